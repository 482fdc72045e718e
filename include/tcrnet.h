/*
 * tcrnet — B300 (sm_103a) builder of the CDR3beta similarity network of
 * "Large-scale GPU-based network analysis of the human T-cell receptor
 * repertoire" (arXiv 2112.06613, TCR-NET).
 *
 * The network (Methods "TCR network"): one node per input string; an undirected
 * edge joins nodes i != j iff the Levenshtein distance of their strings
 * (Methods "Levenshtein distance", Eq. levenshtein: unit-cost insertion,
 * deletion and substitution) does not exceed the threshold l_max. It is
 * returned as the rows of the symmetric 0/1 adjacency matrix (Methods
 * "Adjacency matrix") in CSR form: row i lists every neighbour j in strictly
 * ascending order, both directions stored, no self-loops; degree[i] =
 * offsets[i+1] - offsets[i] (d(u) = sum_v A_uv, Methods "Overview of network
 * theory concepts").
 *
 * Conventions shared by every entry point:
 *  - Strings are upper-case one-letter codes of the 20 standard amino acids
 *    (the set Sigma of Methods "Combination of amino acids"), length 1 ..
 *    TCRNET_MAX_LEN. Anything else is rejected (TCRNET_EBADCHAR,
 *    TCRNET_ETOOLONG, TCRNET_EINVAL for an empty string); strings are never
 *    truncated, since truncation changes distances. The offending input index
 *    is then available from tcrnet_last_error_index().
 *  - Node id = input position. Duplicate strings are distinct nodes and are
 *    adjacent to each other (distance 0).
 *  - Inputs are borrowed for the duration of the call and never retained.
 *  - Thresholds: any l_max >= 0 (negative: TCRNET_EINVAL). 0 and 1 (the paper's
 *    network-construction setting, Fig. performance) use closed-form tests or
 *    the deletion join; 2 (the paper's assortativity analysis) uses the
 *    deletion method's candidates (strings sharing a variant with up to two
 *    deletions) checked by the exact bit-parallel distance, or the all-pairs
 *    distance kernel for small inputs; l_max >= 3 (the paper's LCC drawings use
 *    6) computes the distance bit-parallel on the tile path
 *    (TCRNET_METHOD_DELETION with l_max >= 3: TCRNET_ENOTSUP).
 *  - Work is ordered on the CUDA stream given in tcrnet_options (NULL: the
 *    legacy default stream). Calls return after the result is complete on the
 *    device unless stated otherwise.
 *  - A handle is thread-compatible, not thread-safe: do not use one handle
 *    from two host threads at once.
 *  - TCRNET_EDEVICE poisons the handle being built or used; free it. The only
 *    bounded device loop (the union-find of tcrnet_components) reports running
 *    out as TCRNET_ETIMEOUT and leaves the handle usable. No call leaves a
 *    sticky device error behind on purpose.
 *  - Memory spaces: arguments tagged `mem` are TCRNET_HOST (pageable or pinned
 *    host memory) or TCRNET_DEVICE (device memory of the handle's device).
 */
#ifndef TCRNET_H
#define TCRNET_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Longest accepted string. The paper reserves 30 amino acids per sequence on
 * the GPU (Methods "GPU-based network generation"); this library accepts up to
 * 48 (two 128-bit words of 5-bit codes). */
#define TCRNET_MAX_LEN 48

typedef enum tcrnet_status {
    TCRNET_OK = 0,
    TCRNET_EINVAL = 1,    /* bad argument, empty string or non-monotone offsets */
    TCRNET_EBADCHAR = 2,  /* a character outside the 20-letter alphabet */
    TCRNET_ETOOLONG = 3,  /* a string longer than TCRNET_MAX_LEN */
    TCRNET_ENOTSUP = 4,   /* combination not supported (deletion method with l_max >= 3, ...) */
    TCRNET_ENOMEM = 5,    /* device or host allocation failed; nothing leaked */
    TCRNET_EDEVICE = 6,   /* a CUDA error; the handle is poisoned */
    TCRNET_ETIMEOUT = 7,  /* a bounded device loop ran out (analytics; the handle stays usable) */
    TCRNET_ESTATE = 8,    /* the handle cannot serve this call (e.g. query on a query result) */
    TCRNET_ECAPACITY = 9  /* input larger than a fixed-capacity entry point accepts */
} tcrnet_status;

typedef enum tcrnet_method {
    TCRNET_METHOD_AUTO = 0,     /* the library picks (deletion path above a size cut-over) */
    TCRNET_METHOD_TILE = 1,     /* all-pairs tile kernel over length buckets */
    TCRNET_METHOD_DELETION = 2  /* deletion-neighbourhood join */
} tcrnet_method;

typedef enum tcrnet_memspace { TCRNET_HOST = 0, TCRNET_DEVICE = 1 } tcrnet_memspace;

/* Options. Fill with tcrnet_options_init, then set what you need; a NULL
 * options pointer means the defaults. */
typedef struct tcrnet_options {
    int32_t method;           /* tcrnet_method (default AUTO) */
    int32_t device;           /* CUDA device ordinal; -1 (default) = the calling
                                 thread's current device */
    int32_t force_offsets64;  /* 1: export int64 offsets even when nnz < 2^31 */
    void *stream;             /* cudaStream_t; NULL = legacy default stream */
    int32_t profile;          /* 1: record per-phase CUDA-event times (tcrnet_stats) */
    int32_t partition_cap;    /* testing: deletion-join partitions larger than this
                                 take the quadratic join pass; 0 = default */
    int32_t partition_target; /* tuning: mean records per deletion-join partition,
                                 4 .. 128; 0 = default (12 up to 2^25 records,
                                 else 32). Any value gives the same network. */
    int32_t fail_alloc_at;    /* testing (host-side fault injection): the k-th device
                                 allocation of this call fails and the call returns
                                 TCRNET_ENOMEM after releasing what it holds;
                                 0 = off */
    int32_t insert_rebuild;   /* inserts (tcrnet_insert_ex, tcrnet_extend): 1 = rebuild
                                 the grown repertoire from scratch; 2 = merge the new
                                 strings into the handle's network and index whenever
                                 the index can take them (deletion builds with
                                 l_max = 1, partitions not overfull); 0 (default) =
                                 merge where that is the faster of the two (measured
                                 rule: see tcrnet_insert_flat). Every way gives the
                                 same network; other values: TCRNET_EINVAL */
    int32_t link_attempts;    /* testing (tcrnet_components_ex): attempts each edge of
                                 the union-find may make to link its two roots before
                                 the call gives up with TCRNET_ETIMEOUT; 0 = default
                                 (2^20, never reached in practice) */
    int32_t deletion_max_n;   /* testing: largest repertoire the deletion method takes;
                                 0 = default (TCRNET_DELETION_MAX_N). AUTO builds
                                 larger repertoires with the tile method; an explicit
                                 TCRNET_METHOD_DELETION above it is TCRNET_ENOTSUP */
    int32_t record_hash_bits; /* testing: the deletion join keeps only this many low
                                 bits (1 .. 31) of each record's 32-bit content hash,
                                 so that variants of different contents match and
                                 the join's confirmation by content has candidates
                                 to reject; such a build keeps no query index.
                                 0 = default (all 32 bits). Any value gives the same
                                 network. */
    int32_t reserved[1];      /* must be zero */
} tcrnet_options;

/* Largest repertoire of the deletion method (distinct-string ids take 25 bits
 * of a join record). Larger inputs are built by the tile method under AUTO. */
#define TCRNET_DELETION_MAX_N (1 << 25)

/* Defaults: AUTO method, current device, legacy default stream, no profiling. */
void tcrnet_options_init(tcrnet_options *opt);

/* Per-build counters and (with options.profile) CUDA-event phase times, all in
 * milliseconds measured on the build's stream. */
typedef struct tcrnet_stats {
    int32_t method;           /* tcrnet_method actually used */
    int32_t threshold;
    int64_t n;                /* nodes */
    int64_t nnz;              /* directed entries = 2 |E| */
    int64_t candidate_pairs;  /* unordered pairs the tile kernel tested (tile path);
                                 deletion path at l_max = 2: string pairs sharing a
                                 variant, checked with the exact distance */
    int64_t n_unique;         /* distinct strings (deletion path) */
    int64_t n_records;        /* deletion-join records (deletion path) */
    int64_t unique_edges;     /* edges among distinct strings (deletion path) */
    int64_t n_fallback;       /* deletion-join partitions over the warp capacity
                                 (joined by the quadratic pass) */
    int64_t kernel_launches;  /* CUDA kernels this call launched */
    int64_t closed_total;     /* deletion path: sum over distinct strings of |closed neighbourhood| */
    int64_t two_pass_join;    /* deletion path: 1 if the edges overflowed the one-pass buffer */
    double ms_upload;         /* host -> device copy of the input (host inputs only) */
    double ms_pack;           /* validate, encode, bucket */
    double ms_count;          /* tile count pass / deletion join count */
    double ms_scan;           /* offsets */
    double ms_write;          /* tile write pass / deletion fill */
    double ms_sort;           /* per-row ordering */
    double ms_total;          /* whole call on the stream */
    double ms_phase[8];       /* deletion path sub-phases: dedup, records, join (weighted
                                 degrees), list sizes + fill, unused, list sort, expand,
                                 total */
    int64_t merged_inserts;   /* inserts merged into this network since its last
                                 full build (0 after a build or a rebuild) */
    int64_t rejected_candidates; /* deletion path, l_max = 1: candidate pairs of equal
                                    32-bit hash whose contents differ (rejected by the
                                    confirmation; hash collisions) */
} tcrnet_stats;

/* Opaque handle: a CSR (n rows) owned by the library in device memory, plus,
 * for a build, the packed resident repertoire that tcrnet_query searches. */
typedef struct tcrnet_graph *tcrnet_handle;

/*
 * Build the network of n strings given as NUL-terminated C strings (host
 * memory). threshold = l_max. On success *out receives a new handle (free it
 * with tcrnet_free); on failure *out is set to NULL.
 */
tcrnet_status tcrnet_build(const char *const *seqs, int64_t n, int32_t threshold,
                           const tcrnet_options *opt, tcrnet_handle *out);

/*
 * Build from a flat layout: chars holds all strings back to back (no
 * separators), offsets has n + 1 entries and string i is
 * chars[offsets[i] .. offsets[i+1]). offsets[0] need not be 0. Both arrays live
 * in memory space `mem`. With TCRNET_HOST the upload is part of the call.
 */
tcrnet_status tcrnet_build_flat(const uint8_t *chars, const int64_t *offsets, int64_t n,
                                int32_t mem, int32_t threshold, const tcrnet_options *opt,
                                tcrnet_handle *out);

/*
 * Batched build: the networks of nrep independent repertoires in one pass.
 * The n strings (flat layout in memory space `mem`) are the repertoires back to
 * back; repertoire r is strings rep_offsets[r] .. rep_offsets[r+1]
 * (rep_offsets: nrep + 1 int64 in HOST memory, rep_offsets[0] = 0,
 * rep_offsets[nrep] = n, non-decreasing, nrep <= 65536). The handle holds one
 * block-diagonal CSR: row i of repertoire r lists the global ids of i's
 * neighbours within r, so rows rep_offsets[r] .. rep_offsets[r+1] minus
 * rep_offsets[r] are exactly the network tcrnet_build_flat would return for
 * that repertoire alone. l_max <= 2 (deletion method; ENOTSUP otherwise or with
 * TCRNET_METHOD_TILE). Batched handles answer no queries or inserts (ESTATE).
 */
tcrnet_status tcrnet_build_batched(const uint8_t *chars, const int64_t *offsets, int64_t n,
                                   const int64_t *rep_offsets, int64_t nrep, int32_t mem, int32_t threshold,
                                   const tcrnet_options *opt, tcrnet_handle *out);

/*
 * Checkpoint / resume of a serving state. tcrnet_save writes a build handle
 * (network, resident strings and, for deletion builds, the query index) to the
 * file `path` (host byte order, format version 3); tcrnet_load makes a new
 * handle from such a file on opt->device / opt->stream (opt may be NULL) that
 * answers queries and inserts like the saved one. Errors: TCRNET_EINVAL (NULL
 * argument, unreadable or unwritable file, bad magic, version or sizes; the
 * header is checked before any device work), TCRNET_ESTATE (query results are
 * not saved), TCRNET_ENOMEM / TCRNET_EDEVICE.
 */
tcrnet_status tcrnet_save(tcrnet_handle h, const char *path);
tcrnet_status tcrnet_load(const char *path, const tcrnet_options *opt, tcrnet_handle *out);

/* Size of a handle's CSR: rows, directed entries (nnz = sum of degrees) and
 * whether exported offsets are int64 (nnz >= 2^31 or force_offsets64). Any
 * pointer may be NULL. */
tcrnet_status tcrnet_info(tcrnet_handle h, int64_t *n, int64_t *nnz, int32_t *offsets_are_64bit);

/*
 * Copy the CSR into caller-owned buffers in memory space `mem`:
 * offsets (n + 1 entries, int32 or int64 as tcrnet_info reports), cols (nnz
 * int32), degree (n int32). Any of the three may be NULL to skip it.
 */
tcrnet_status tcrnet_copy_csr(tcrnet_handle h, void *offsets, int32_t *cols, int32_t *degree,
                              int32_t mem);

/* Device pointers of the CSR, owned by the handle and valid until tcrnet_free.
 * Any output pointer may be NULL. */
tcrnet_status tcrnet_csr_device(tcrnet_handle h, const void **offsets, const int32_t **cols,
                                const int32_t **degree);

/*
 * Neighbour lists of m query strings against the resident repertoire of a
 * build handle: for query q, every node j with lev(query_q, s_j) <= the build's
 * threshold, ascending. A query equal to a node's string lists that node (a
 * query is not a node, so nothing is excluded). Flat layout as in
 * tcrnet_build_flat. *out receives a new handle whose CSR has m rows (query it
 * with tcrnet_info / tcrnet_copy_csr; it cannot itself be queried).
 */
tcrnet_status tcrnet_query_flat(tcrnet_handle h, const uint8_t *chars, const int64_t *offsets,
                                int64_t m, int32_t mem, tcrnet_handle *out);

/* tcrnet_query_flat with options: opt->stream orders the call (NULL options or
 * stream: the build's stream); opt->method selects the search: AUTO (the
 * deletion index when the build kept one, i.e. a deletion-method build with
 * l_max = 1 or 2, else the tile kernel), TILE, or DELETION (ENOTSUP without an
 * index). Both searches return identical lists. The l_max = 2 index holds the
 * variant records of the build (every distinct string with up to two
 * deletions); a query looks up its own variants and checks each distinct
 * candidate with the exact distance. */
tcrnet_status tcrnet_query_ex(tcrnet_handle h, const uint8_t *chars, const int64_t *offsets, int64_t m,
                              int32_t mem, const tcrnet_options *opt, tcrnet_handle *out);

/* Same as tcrnet_query_flat for NUL-terminated host strings. */
tcrnet_status tcrnet_query(tcrnet_handle h, const char *const *queries, int64_t m,
                           tcrnet_handle *out);

/*
 * Append m strings to a build handle as nodes n .. n+m-1 (flat layout as in
 * tcrnet_build_flat). On success the handle's CSR, degree, resident repertoire
 * and query index describe the grown repertoire, exactly as a fresh build of
 * the concatenated input would (node ids of existing strings are unchanged);
 * previously returned device pointers (tcrnet_csr_device) become invalid. The
 * update is computed on the device from the handle's packed strings: a deletion
 * build (l_max = 1) merges the new strings into its network and query index
 * (the new strings' closed neighbourhoods from a query of the grown index, old
 * rows grown at their ends) where that is faster than a rebuild, by a rule
 * measured on a B300: from 7e5 resident strings for inserts of up to n/2048,
 * from 1.5e6 for inserts of up to n/32; other inserts rebuild the grown
 * repertoire (options.insert_rebuild forces either way). Both give the network
 * of a fresh build of the concatenation. On failure
 * (bad string: its index within the new batch is reported) the handle keeps its
 * previous network. Not for query-result handles (ESTATE). Callers must not use
 * the handle from another thread during the call.
 */
tcrnet_status tcrnet_insert_flat(tcrnet_handle h, const uint8_t *chars, const int64_t *offsets, int64_t m,
                                 int32_t mem);

/* tcrnet_insert_flat with options (opt->stream orders the call; opt->profile). */
tcrnet_status tcrnet_insert_ex(tcrnet_handle h, const uint8_t *chars, const int64_t *offsets, int64_t m,
                               int32_t mem, const tcrnet_options *opt);

/* tcrnet_insert_flat for NUL-terminated host strings. */
tcrnet_status tcrnet_insert(tcrnet_handle h, const char *const *seqs, int64_t m);

/*
 * Copy-on-write insert: a NEW handle whose network is that of h's strings
 * followed by the m new strings (ids n, n+1, ... as with tcrnet_insert); h is
 * not modified and only read, so queries on h may continue on other host
 * threads and streams while the new network is built (h's reads are of memory
 * that no call modifies). The caller swaps handles when it returns and frees
 * the old one after its last query. Same arguments and errors as
 * tcrnet_insert_ex; on error *out = NULL. m = 0 gives a rebuilt copy.
 */
tcrnet_status tcrnet_extend(tcrnet_handle h, const uint8_t *chars, const int64_t *offsets, int64_t m, int32_t mem,
                            const tcrnet_options *opt, tcrnet_handle *out);

/*
 * Connected components of the network restricted to the nodes with keep[i] != 0
 * (keep == NULL keeps every node): node removal of the robustness analysis
 * (Methods "Computing LCC"; the caller draws which nodes are removed). labels
 * (n int32, may be NULL) receives the smallest node id of each node's component,
 * -1 for removed nodes; *n_components the number of components among kept
 * nodes; *largest the size of the largest one (LCC). keep and labels live in
 * memory space `mem`. TCRNET_ETIMEOUT if the bounded union retry loop ran out
 * (not expected; the handle stays usable).
 */
tcrnet_status tcrnet_components(tcrnet_handle h, const uint8_t *keep, int32_t *labels, int32_t mem,
                                int64_t *n_components, int64_t *largest);

/* tcrnet_components with options: opt->stream orders the call (NULL options or
 * stream: the handle's stream); opt->link_attempts bounds the attempts of each
 * edge to link its two roots (testing; 0 = default). When an edge runs out of
 * attempts the kernel records it and returns, every other edge is still
 * processed, and the call reports TCRNET_ETIMEOUT with *n_components and
 * *largest set to 0; labels are then undefined. The handle and the device stay
 * usable: nothing waits without a bound. */
tcrnet_status tcrnet_components_ex(tcrnet_handle h, const uint8_t *keep, int32_t *labels, int32_t mem,
                                   const tcrnet_options *opt, int64_t *n_components, int64_t *largest);

/* Average neighbour degree (Methods "Overview of network theory concepts",
 * <d_nn>): knn[i] = (sum over neighbours j of d(j)) / d(i), 0 for isolated nodes;
 * n doubles in memory space `mem`. */
tcrnet_status tcrnet_neighbor_degree(tcrnet_handle h, double *knn, int32_t mem);

/* Degree distribution (Results, degree distributions of the networks; d(u) of
 * Methods "Overview of network theory concepts"): hist[d] = number of nodes of
 * degree d for d < nbins - 1; hist[nbins - 1] counts every node of degree >=
 * nbins - 1. nbins >= 1 int64 counters in memory space `mem`. *max_degree (may
 * be NULL) receives the largest degree, so a caller can size the bins exactly. */
tcrnet_status tcrnet_degree_histogram(tcrnet_handle h, int64_t *hist, int64_t nbins, int32_t mem,
                                      int64_t *max_degree);

/* Counters and phase times of the call that produced the handle. */
tcrnet_status tcrnet_stats_get(tcrnet_handle h, tcrnet_stats *out);

/* Release a handle and all device memory it owns. NULL is a no-op. The memory
 * is returned stream-ordered without waiting for the device; finish any work of
 * your own that reads the handle's device pointers before freeing it. */
void tcrnet_free(tcrnet_handle h);

/* Static description of a status code. */
const char *tcrnet_strerror(tcrnet_status s);

/* Input index that caused the calling thread's most recent EBADCHAR /
 * ETOOLONG / EINVAL, or -1. */
int64_t tcrnet_last_error_index(void);

/* Library version string. */
const char *tcrnet_version(void);

/* Text of the calling thread's last failing CUDA call (diagnostics; "" if none). */
const char *tcrnet_last_cuda_error(void);

/* Largest n tcrnet_degree_noalloc accepts. */
#define TCRNET_NOALLOC_MAX_N 16384

/*
 * Node degrees of the network of at most TCRNET_NOALLOC_MAX_N strings, without
 * allocating any memory. The paper has no counterpart: this entry point exists
 * for callers that cannot call cudaMalloc. Two kinds of program are in that
 * position: one whose device memory has been handed in full, at start-up, to
 * another allocator (a framework's caching pool that reserves all free memory,
 * so a new allocation fails or would have to evict its cache), and one that
 * forbids device allocation after start-up to keep its latency bounded (an
 * allocation can synchronise the device or map new pages). Every other entry
 * point allocates its workspace and results itself.
 *
 * d_chars / d_offsets: the flat string layout of tcrnet_build_flat, in device
 * memory of the calling thread's current device. d_degree: device output of n
 * int32, overwritten with d(i) = number of j != i with lev(s_i, s_j) <=
 * threshold (threshold 0 or 1); equal to tcrnet_copy_csr's degree for the same
 * input. stream: cudaStream_t (NULL = legacy default stream). bad_index
 * (optional host pointer) receives the offending input index on
 * EBADCHAR / ETOOLONG / EINVAL, else -1. The call returns when the result is
 * complete.
 *
 * Errors: TCRNET_ECAPACITY if n > TCRNET_NOALLOC_MAX_N (nothing runs);
 * EINVAL / ENOTSUP for bad arguments; EBADCHAR / ETOOLONG / EINVAL for bad
 * strings; EDEVICE for a CUDA error.
 *
 * Working memory is one fixed file-scope device array of about 0.5 MB that
 * every device loading the library keeps until the process exits. The first
 * call on each device looks up that array's device address (a one-time set-up
 * step) and keeps it for the life of the process, so make the first call on a
 * device before any stream capture, and do not call this entry point on a
 * device after cudaDeviceReset of that device in the same process (the kept
 * address then refers to the old context). All calls share the array and it
 * keeps the previous call's contents (each call clears what must start at
 * zero), so calls that overlap on the GPU, from different streams or host
 * threads, race: serialise them. The call waits for its stream before
 * returning (it reads back the error word).
 */
tcrnet_status tcrnet_degree_noalloc(const uint8_t *d_chars, const int64_t *d_offsets, int64_t n,
                                    int32_t threshold, int32_t *d_degree, void *stream,
                                    int64_t *bad_index);

/* Kinds of tcrnet_probe_int_issue. */
typedef enum tcrnet_probe_kind {
    TCRNET_PROBE_LOP3 = 0,  /* three-input logic op */
    TCRNET_PROBE_SHF = 1,   /* funnel shift */
    TCRNET_PROBE_IADD = 2,  /* 32-bit add */
    TCRNET_PROBE_IMAD = 3,  /* 32-bit multiply-add */
    TCRNET_PROBE_POPC = 4,  /* xor, population count, add */
    TCRNET_PROBE_MIX = 5    /* logic op, add and multiply-add in turn */
} tcrnet_probe_kind;

/*
 * Integer-issue microbenchmark (a measurement aid; the paper has no
 * counterpart). Launches one kernel on `stream` in which each of n_threads
 * threads (a multiple of 256) runs `iters` rounds of independent dependency
 * chains of 32-bit integer instructions of the given kind and writes one word
 * to d_out[thread] (device memory of the current device, n_threads uint32,
 * caller-owned). *ops_per_thread receives the integer instructions each
 * thread issues in its rounds, so that a caller timing the launch with CUDA
 * events on `stream` gets the per-SM integer rate the all-pairs tile kernel is
 * bound by. Returns without waiting for the kernel. Errors: TCRNET_EINVAL for
 * bad arguments, TCRNET_EDEVICE if the launch fails.
 */
tcrnet_status tcrnet_probe_int_issue(int32_t kind, int32_t iters, uint32_t *d_out, int64_t n_threads,
                                     void *stream, int64_t *ops_per_thread);

/*
 * The per-row ordering step of the builds on its own (the CSR rows are
 * placed in arrival order, then each row is sorted; Methods "Adjacency
 * matrix" gives the matrix the rows stand for). Sorts every row
 * segment d_cols[d_offsets[i] .. d_offsets[i+1]) ascending, in place, for
 * i < n: rows of up to 512 values in registers, up to 16,384 in shared
 * memory, longer ones by shared-memory chunks and stable pairwise merges.
 * Values may repeat (the l_max = 2 candidate rows do). d_offsets: n + 1
 * ascending int64 offsets, d_cols: int32 values, both device memory of the
 * current device, caller-owned; stream: a cudaStream_t or NULL (the legacy
 * default stream). Returns after the sort has finished. Errors: TCRNET_EINVAL
 * for n < 0 or null pointers with n > 0, TCRNET_ENOMEM if scratch memory
 * cannot be had, TCRNET_EDEVICE on a device error.
 */
tcrnet_status tcrnet_sort_rows(const int64_t *d_offsets, int32_t *d_cols, int64_t n, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* TCRNET_H */
