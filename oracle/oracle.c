/*
 * CPU oracle for the TCR network (test infrastructure only).
 *
 * Only the test suite, the smoke check and the bench's CPU-baseline leg load
 * this library. The product path (the CUDA library) never links, calls or
 * falls back to it, and the two share no code.
 *
 * What it computes, from the paper:
 *   - lev(a, b): the unit-cost edit distance of the Levenshtein recurrence
 *     (Methods "Levenshtein distance", Eq. levenshtein, with the indicator
 *     1(a_i != b_j)), evaluated iteratively as the textbook Wagner-Fischer
 *     table kept as two rows. No early exit, no length filter.
 *   - The TCR network (Methods "TCR network"): node i per input string, an
 *     undirected edge {i, j}, i != j, iff lev(s_i, s_j) <= l_max.
 *   - Serialised as the rows of the adjacency matrix (Methods "Adjacency
 *     matrix"): row i lists every j with A_ij = 1 in ascending order; the
 *     degree d(i) is the row length (Methods "Overview of network theory
 *     concepts", d(u) = sum_v A_uv).
 *
 * Readings where the paper is ambiguous:
 *   - base case: lev of a prefix against the empty prefix is the prefix
 *     length (the recurrence's "max(i-1, j-1) if i = 1 or j = 1" with 1-based
 *     indices, where index 1 denotes the empty prefix);
 *   - edge rule "does not exceed l_max", i.e. lev <= l_max (Introduction and
 *     Methods "TCR network"); the pseudocode listing's strict "<" is not used;
 *   - duplicates are separate nodes; identical strings are adjacent (lev 0);
 *     no self-loops (the zero diagonal of the adjacency example).
 *
 * Queries use the same rule against a repertoire: for each query q, all j with
 * lev(q, s_j) <= l_max, ascending, excluding self_index[q] when it is >= 0
 * (row i of the network is the query s_i with self index i).
 *
 * Strings are arbitrary byte strings here; alphabet checks belong to the
 * library under test, not to the definition.
 *
 * The file also holds the CPU baseline of the bench (baseline_within,
 * baseline_neighbors: the paper's early-abort algorithm); it is not used as the
 * oracle, and the test suite pins its answers to oracle_lev.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int min3(int x, int y, int z) {
    int m = x < y ? x : y;
    return m < z ? m : z;
}

/* lev(a, b) by the Wagner-Fischer table, two rows of length lb + 1.
 * prev[j] holds lev(a[0..i-1), b[0..j)) and cur[j] holds lev(a[0..i), b[0..j)). */
int oracle_lev(const uint8_t *a, int64_t la, const uint8_t *b, int64_t lb) {
    int stackbuf[2 * 130];
    int *buf = stackbuf;
    if (lb + 1 > 130) {
        buf = (int *)malloc(sizeof(int) * 2 * (size_t)(lb + 1));
        if (!buf) return -1;
    }
    int *prev = buf;
    int *cur = buf + (lb + 1);
    for (int64_t j = 0; j <= lb; ++j) prev[j] = (int)j; /* lev(empty, b[0..j)) = j */
    for (int64_t i = 1; i <= la; ++i) {
        cur[0] = (int)i; /* lev(a[0..i), empty) = i */
        for (int64_t j = 1; j <= lb; ++j) {
            int ind = (a[i - 1] != b[j - 1]) ? 1 : 0; /* 1(a_i != b_j) */
            cur[j] = min3(prev[j] + 1,          /* deletion of a_i  */
                          cur[j - 1] + 1,       /* insertion of b_j */
                          prev[j - 1] + ind);   /* match / substitution */
        }
        int *t = prev;
        prev = cur;
        cur = t;
    }
    int d = prev[lb];
    if (buf != stackbuf) free(buf);
    return d;
}

/* Row lists of one query against the repertoire. */
typedef struct {
    int64_t len, cap;
    int32_t *v;
} ivec;

static int ivec_push(ivec *x, int32_t val) {
    if (x->len == x->cap) {
        int64_t nc = x->cap ? 2 * x->cap : 16;
        int32_t *nv = (int32_t *)realloc(x->v, sizeof(int32_t) * (size_t)nc);
        if (!nv) return -1;
        x->v = nv;
        x->cap = nc;
    }
    x->v[x->len++] = val;
    return 0;
}

typedef struct oracle_lists {
    int64_t rows;
    int64_t nnz;
    int64_t *offsets; /* rows + 1 */
    int32_t *cols;    /* nnz */
} oracle_lists;

/* Concatenate m row lists into one CSR and free them; NULL if `failed` or on
 * allocation failure. */
static oracle_lists *lists_from_rows(ivec *rows, int64_t m, int failed) {
    oracle_lists *out = (oracle_lists *)calloc(1, sizeof(oracle_lists));
    if (out) {
        out->rows = m;
        out->offsets = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m + 1));
        int64_t total = 0;
        for (int64_t q = 0; q < m; ++q) total += rows[q].len;
        out->nnz = total;
        out->cols = (int32_t *)malloc(sizeof(int32_t) * (size_t)(total > 0 ? total : 1));
        if (!out->offsets || !out->cols) failed = 1;
        if (!failed) {
            int64_t o = 0;
            for (int64_t q = 0; q < m; ++q) {
                out->offsets[q] = o;
                if (rows[q].len) memcpy(out->cols + o, rows[q].v, sizeof(int32_t) * (size_t)rows[q].len);
                o += rows[q].len;
            }
            out->offsets[m] = o;
        }
    }
    for (int64_t q = 0; q < m; ++q) free(rows[q].v);
    free(rows);
    if (failed && out) {
        free(out->offsets);
        free(out->cols);
        free(out);
        out = NULL;
    }
    return out;
}

/*
 * For each query q in [0, m): every repertoire index j in [0, n), ascending,
 * with j != self_index[q] and lev(query_q, s_j) <= max_dist.
 * self_index may be NULL (no exclusion). nthreads <= 0 uses the OpenMP default.
 * Returns NULL on allocation failure.
 */
oracle_lists *oracle_neighbors(const uint8_t *chars, const int64_t *offsets, int64_t n,
                               const uint8_t *qchars, const int64_t *qoffsets, int64_t m,
                               const int64_t *self_index, int32_t max_dist, int32_t nthreads) {
    ivec *rows = (ivec *)calloc((size_t)(m > 0 ? m : 1), sizeof(ivec));
    if (!rows) return NULL;
    int failed = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < m; ++q) {
        const uint8_t *a = qchars + qoffsets[q];
        int64_t la = qoffsets[q + 1] - qoffsets[q];
        int64_t self = self_index ? self_index[q] : -1;
        for (int64_t j = 0; j < n; ++j) {
            if (j == self) continue;
            int d = oracle_lev(a, la, chars + offsets[j], offsets[j + 1] - offsets[j]);
            if (d < 0) {
                failed = 1;
                break;
            }
            if (d <= max_dist) {
                if (ivec_push(&rows[q], (int32_t)j)) {
                    failed = 1;
                    break;
                }
            }
        }
    }
    return lists_from_rows(rows, m, failed);
}

/*
 * CPU BASELINE, not the oracle: the paper's own per-pair test (Methods
 * "GPU-based network generation" and its Listing 1), restated correctly, for
 * the timed CPU baseline of the bench. It answers "lev(a, b) <= max_dist?"
 * with the same two-row table as oracle_lev, filled one row of `a` at a time,
 * and stops as soon as every entry of the finished row exceeds max_dist: the
 * smallest entry of a row never decreases from one row to the next (each entry
 * extends an entry of the row above by a non-negative cost, or the entry to its
 * left, whose chain starts at the row's first column i >= i - 1), so the final
 * distance would exceed max_dist as well. Pairs whose lengths differ by more
 * than max_dist are answered without a table, because the distance is at least
 * the difference of the lengths. The answer equals oracle_lev(...) <= max_dist
 * for every pair (pinned by the test suite); only the work differs.
 */
int baseline_within(const uint8_t *a, int64_t la, const uint8_t *b, int64_t lb, int32_t max_dist) {
    int64_t dl = la > lb ? la - lb : lb - la;
    if (dl > max_dist) return 0;
    int stackbuf[2 * 130];
    int *buf = stackbuf;
    if (lb + 1 > 130) {
        buf = (int *)malloc(sizeof(int) * 2 * (size_t)(lb + 1));
        if (!buf) return -1;
    }
    int *row = buf;            /* row i - 1 of the table */
    int *next = buf + (lb + 1); /* row i */
    for (int64_t j = 0; j <= lb; ++j) row[j] = (int)j;
    int within = 1;
    for (int64_t i = 1; i <= la; ++i) {
        next[0] = (int)i;
        int row_min = next[0];
        for (int64_t j = 1; j <= lb; ++j) {
            int sub = row[j - 1] + ((a[i - 1] == b[j - 1]) ? 0 : 1);
            int del = row[j] + 1;
            int ins = next[j - 1] + 1;
            int v = sub < del ? sub : del;
            v = v < ins ? v : ins;
            next[j] = v;
            if (v < row_min) row_min = v;
        }
        int *t = row;
        row = next;
        next = t;
        if (row_min > max_dist) { /* early abort: no later row can come back under the bound */
            within = 0;
            break;
        }
    }
    if (within) within = row[lb] <= max_dist;
    if (buf != stackbuf) free(buf);
    return within;
}

/*
 * The network rows of the queries by baseline_within (same contract and
 * output as oracle_neighbors; nthreads = 1 gives the single-core baseline).
 */
oracle_lists *baseline_neighbors(const uint8_t *chars, const int64_t *offsets, int64_t n,
                                 const uint8_t *qchars, const int64_t *qoffsets, int64_t m,
                                 const int64_t *self_index, int32_t max_dist, int32_t nthreads) {
    ivec *rows = (ivec *)calloc((size_t)(m > 0 ? m : 1), sizeof(ivec));
    if (!rows) return NULL;
    int failed = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < m; ++q) {
        const uint8_t *a = qchars + qoffsets[q];
        int64_t la = qoffsets[q + 1] - qoffsets[q];
        int64_t self = self_index ? self_index[q] : -1;
        for (int64_t j = 0; j < n; ++j) {
            if (j == self) continue;
            int w = baseline_within(a, la, chars + offsets[j], offsets[j + 1] - offsets[j], max_dist);
            if (w < 0) {
                failed = 1;
                break;
            }
            if (w && ivec_push(&rows[q], (int32_t)j)) {
                failed = 1;
                break;
            }
        }
    }
    return lists_from_rows(rows, m, failed);
}

int64_t oracle_lists_rows(const oracle_lists *l) { return l->rows; }
int64_t oracle_lists_nnz(const oracle_lists *l) { return l->nnz; }

void oracle_lists_copy(const oracle_lists *l, int64_t *offsets, int32_t *cols) {
    memcpy(offsets, l->offsets, sizeof(int64_t) * (size_t)(l->rows + 1));
    if (l->nnz) memcpy(cols, l->cols, sizeof(int32_t) * (size_t)l->nnz);
}

void oracle_lists_free(oracle_lists *l) {
    if (!l) return;
    free(l->offsets);
    free(l->cols);
    free(l);
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
