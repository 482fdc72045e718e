// C ABI and host runtime of tcrnet (declarations and contracts: include/tcrnet.h).
//
// A build runs: upload (host inputs only) -> pack (validate, encode, bucket) ->
// the chosen method (tile: count pass, offsets, write pass, row sort;
// deletion: deletion.cu) -> export (int32 or int64 offsets, degree). The
// result stays in device memory owned by the handle; host copies happen only
// in tcrnet_copy_csr.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "deletion.cuh"
#include "kernels.cuh"

struct tcrnet_graph {
    int device = 0;
    cudaStream_t stream = 0;
    bool query_result = false;
    bool batched = false;  // block-diagonal network of several repertoires
    int32_t threshold = 1;
    int64_t n = 0;
    int64_t nnz = 0;
    int offsets64 = 0;
    void* d_offsets = nullptr;
    int32_t* d_cols = nullptr;
    int32_t* d_degree = nullptr;
    // resident repertoire (build handles only): the bucketed copy (tile
    // builds) or the input-order copy (deletion builds), and the total length
    tcr::Canon* d_bcanon = nullptr;
    int32_t* d_bperm = nullptr;
    int64_t bucket_off[tcr::kMaxLen + 2] = {0};
    tcr::Canon* d_canon_in = nullptr;
    uint8_t* d_lens = nullptr;
    int64_t lensum = 0;
    tcr::DeletionIndex ix;  // query index of a deletion build (l_max >= 1)
    tcrnet_stats stats;
};

namespace tcr {

static thread_local int64_t t_last_bad = -1;
static thread_local int64_t t_launches = 0;

void note_launch() { ++t_launches; }

static thread_local int64_t t_alloc_countdown = -1;  // -1: fault injection off

bool alloc_fault_tick() {
    if (t_alloc_countdown < 0) return false;
    if (t_alloc_countdown == 0) return true;  // stays armed: later allocations fail too
    --t_alloc_countdown;
    return t_alloc_countdown == 0;
}

AllocFaultScope::AllocFaultScope(int32_t fail_at) : saved_(t_alloc_countdown) {
    t_alloc_countdown = fail_at > 0 ? (int64_t)fail_at : -1;
}

AllocFaultScope::~AllocFaultScope() { t_alloc_countdown = saved_; }
int64_t launches_so_far() { return t_launches; }

// ---- build workspace arena (see common.cuh) ----
namespace {
constexpr size_t kArenaAlign = 256;
constexpr size_t kMinChunk = 64ull << 20;
struct Chunk {
    char* p;
    size_t size;
};
struct DeviceArena {
    std::mutex mu;
    std::vector<Chunk> chunks;
    size_t cur = 0;   // chunk being carved
    size_t used = 0;  // bytes used in chunks[cur]
    SideStream side;  // created on first use, kept for the process
    bool side_ok = false;
};
DeviceArena g_arenas[64];
thread_local DeviceArena* t_arena = nullptr;
}  // namespace

bool arena_active() { return t_arena != nullptr; }

namespace {
struct PinnedScratch {
    void* p = nullptr;
    void* dev = nullptr;
    bool tried = false;
    ~PinnedScratch() {
        if (p) cudaFreeHost(p);  // at process exit the runtime may be gone: the error is ignored
    }
};
thread_local PinnedScratch t_pinned;
}  // namespace

void* pinned_scratch() {
    if (!t_pinned.tried) {
        t_pinned.tried = true;
        if (cudaHostAlloc(&t_pinned.p, kPinnedScratchBytes, cudaHostAllocPortable | cudaHostAllocMapped) !=
            cudaSuccess) {
            t_pinned.p = nullptr;
            (void)cudaGetLastError();
        } else if (cudaHostGetDevicePointer(&t_pinned.dev, t_pinned.p, 0) != cudaSuccess) {
            t_pinned.dev = nullptr;
            (void)cudaGetLastError();
        }
    }
    return t_pinned.p;
}

void* pinned_scratch_device() {
    return pinned_scratch() ? t_pinned.dev : nullptr;
}

tcrnet_status read_back(cudaStream_t s, int count, const void* const* src, void* const* dst, const size_t* bytes) {
    size_t total = 0;
    for (int k = 0; k < count; ++k) total += (bytes[k] + 15) & ~size_t(15);
    uint8_t* pin = static_cast<uint8_t*>(pinned_scratch());
    if (!pin || total > kPinnedScratchBytes) {
        for (int k = 0; k < count; ++k)
            TCR_CUDA(cudaMemcpyAsync(dst[k], src[k], bytes[k], cudaMemcpyDeviceToHost, s));
        TCR_CUDA(cudaStreamSynchronize(s));
        return TCRNET_OK;
    }
    size_t at = 0;
    for (int k = 0; k < count; ++k) {
        TCR_CUDA(cudaMemcpyAsync(pin + at, src[k], bytes[k], cudaMemcpyDeviceToHost, s));
        at += (bytes[k] + 15) & ~size_t(15);
    }
    TCR_CUDA(cudaStreamSynchronize(s));
    at = 0;
    for (int k = 0; k < count; ++k) {
        std::memcpy(dst[k], pin + at, bytes[k]);
        at += (bytes[k] + 15) & ~size_t(15);
    }
    return TCRNET_OK;
}

const SideStream* leased_side_stream() {
    DeviceArena* a = t_arena;
    if (!a) return nullptr;
    if (!a->side_ok) {
        if (cudaStreamCreateWithFlags(&a->side.stream, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
        if (cudaStreamCreateWithFlags(&a->side.stream2, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
        for (auto& e : a->side.ev)
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
        a->side_ok = true;
    }
    return &a->side;
}

namespace {
std::mutex g_event_mu;
std::vector<cudaEvent_t> g_event_pool[64];
}  // namespace

cudaEvent_t event_acquire() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    {
        std::lock_guard<std::mutex> lk(g_event_mu);
        if (!g_event_pool[dev].empty()) {
            cudaEvent_t e = g_event_pool[dev].back();
            g_event_pool[dev].pop_back();
            return e;
        }
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

void event_release(cudaEvent_t e) {
    int dev = 0;
    if (!e || cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        if (e) cudaEventDestroy(e);
        return;
    }
    std::lock_guard<std::mutex> lk(g_event_mu);
    g_event_pool[dev].push_back(e);
}

void* arena_carve(size_t bytes, cudaError_t* err) {
    DeviceArena* a = t_arena;
    if (!a) return nullptr;
    bytes = (bytes + kArenaAlign - 1) & ~(kArenaAlign - 1);
    while (a->cur < a->chunks.size()) {
        Chunk& c = a->chunks[a->cur];
        if (a->used + bytes <= c.size) {
            void* p = c.p + a->used;
            a->used += bytes;
            return p;
        }
        ++a->cur;
        a->used = 0;
    }
    // grow: a new chunk, kept for later calls
    size_t sz = kMinChunk;
    if (!a->chunks.empty()) sz = std::max(sz, a->chunks.back().size * 2);
    sz = std::max(sz, bytes);
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, sz);
    if (e != cudaSuccess) {
        *err = e;
        return nullptr;
    }
    a->chunks.push_back(Chunk{static_cast<char*>(p), sz});
    a->cur = a->chunks.size() - 1;
    a->used = bytes;
    return p;
}

ArenaLease::ArenaLease(int device, cudaStream_t s) : dev_(device), s_(s) {
    if (device < 0 || device >= 64 || t_arena) return;
    DeviceArena& a = g_arenas[device];
    if (!a.mu.try_lock()) return;  // another host thread is building on this device
    held_ = true;
    a.cur = 0;
    a.used = 0;
    t_arena = &a;
}

ArenaLease::~ArenaLease() {
    if (!held_) return;
    // the next lease reuses this memory: the call's work must be complete,
    // on its stream and on the side stream (an early error return may leave
    // forked work there)
    cudaStreamSynchronize(s_);
    if (g_arenas[dev_].side_ok) {
        cudaStreamSynchronize(g_arenas[dev_].side.stream);
        cudaStreamSynchronize(g_arenas[dev_].side.stream2);
    }
    t_arena = nullptr;
    g_arenas[dev_].mu.unlock();
}
static thread_local char t_last_cuda[256] = {0};

void note_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
    std::snprintf(t_last_cuda, sizeof(t_last_cuda), "%s: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
}

namespace {

struct DeviceGuard {
    int prev = -1;
    bool changed = false;
    tcrnet_status set(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) return TCRNET_EDEVICE;
        if (dev >= 0 && dev != prev) {
            if (cudaSetDevice(dev) != cudaSuccess) return TCRNET_EINVAL;
            changed = true;
        }
        return TCRNET_OK;
    }
    ~DeviceGuard() {
        if (changed) cudaSetDevice(prev);
    }
};

// Keep freed stream-ordered allocations cached in the device's default pool
// (a per-process pool attribute), so repeated builds do not return memory to
// the driver and re-map it.
void configure_pool(int dev) {
    static std::mutex mu;
    static bool done[64] = {false};
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 0 || dev >= 64 || done[dev]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    done[dev] = true;
}

// CUDA-event phase timer (active only with options.profile).
using Phases = EventMarks;

int sm_count(int dev) {
    int v = 148;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v;
}

// Per-device non-blocking stream on which handle memory is returned to the
// pool. Every call that touches a handle's memory synchronizes its stream before
// returning, so nothing is pending on it at free time, and a free does not
// serialize work running on other streams (cudaFree would synchronize the device).
cudaStream_t free_stream(int dev) {
    static std::mutex mu;
    static cudaStream_t st[64] = {nullptr};
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 0 || dev >= 64) return 0;
    if (!st[dev] && cudaStreamCreateWithFlags(&st[dev], cudaStreamNonBlocking) != cudaSuccess) st[dev] = 0;
    return st[dev];
}

void free_handle_memory(tcrnet_graph* h) {
    void* ptrs[] = {h->d_offsets, h->d_cols, h->d_degree, h->d_bcanon, h->d_bperm, h->d_canon_in, h->d_lens,
                    h->ix.ucanon, h->ix.umult, h->ix.mem_off, h->ix.members, h->ix.recs, h->ix.poff,
                    h->ix.uid, h->ix.uedges};
    const cudaStream_t fs = free_stream(h->device);
    for (void* p : ptrs)
        if (p) cudaFreeAsync(p, fs);
    h->ix = DeletionIndex();
    h->d_offsets = nullptr;
    h->d_cols = nullptr;
    h->d_degree = nullptr;
    h->d_bcanon = nullptr;
    h->d_bperm = nullptr;
    h->d_canon_in = nullptr;
    h->d_lens = nullptr;
}

// Move a finished CSR (int64 offsets, cols, degree) into the handle, narrowing
// offsets to int32 when they fit.
tcrnet_status export_csr(tcrnet_graph* h, DevBuf& off64, DevBuf& cols, DevBuf& degree, int64_t n, int64_t nnz,
                         bool force64, cudaStream_t s, DevBuf* off32_ready = nullptr) {
    h->n = n;
    h->nnz = nnz;
    h->offsets64 = (force64 || nnz > 0x7fffffffLL) ? 1 : 0;
    if (h->offsets64) {
        h->d_offsets = off64.release();
    } else if (off32_ready && off32_ready->as<void>()) {
        h->d_offsets = off32_ready->release();
    } else {
        DevBuf off32;
        TCR_CHECK(off32.alloc_owned(sizeof(int32_t) * (n + 1), s));
        TCR_CHECK(narrow_offsets(off64.as<int64_t>(), off32.as<int32_t>(), n + 1, s));
        h->d_offsets = off32.release();
    }
    h->d_cols = static_cast<int32_t*>(cols.release());
    h->d_degree = static_cast<int32_t*>(degree.release());
    if (!h->d_offsets || !h->d_cols || !h->d_degree) return TCRNET_EDEVICE;  // scratch cannot be exported
    return TCRNET_OK;
}

// Tile method: count pass -> offsets -> write pass -> row sort.
tcrnet_status tile_method(tcrnet_graph* h, const TileSide& rows, const TileSide& cols, int64_t n_rows, bool sym,
                          int T, bool force64, Phases& ph, cudaStream_t s, int sms) {
    tcrnet_stats& st = h->stats;
    DevBuf count, off64, out_cols, cursor;
    TCR_CHECK(count.alloc_owned(sizeof(int32_t) * n_rows, s));
    TCR_CUDA(cudaMemsetAsync(count.as<void>(), 0, sizeof(int32_t) * n_rows, s));
    // The count pass keeps its hits (up to kPairsPerRow per row on average); when
    // they all fit, a scatter replaces the write pass, which would test every
    // candidate pair again.
    constexpr int64_t kPairsPerRow = 64;
    const int64_t pcap = std::max<int64_t>(1 << 20, std::min<int64_t>(kPairsPerRow * n_rows, 1LL << 28));
    DevBuf pairbuf, pcur;
    PairSink sink;
    if (pairbuf.alloc(sizeof(int2) * pcap, s) == TCRNET_OK && pcur.alloc(sizeof(unsigned long long) * 2, s) == TCRNET_OK) {
        TCR_CUDA(cudaMemsetAsync(pcur.as<void>(), 0, sizeof(unsigned long long) * 2, s));
        sink.pairs = pairbuf.as<int2>();
        sink.cursor = pcur.as<unsigned long long>();
        sink.cap = pcap;
    }
    const int e0 = ph.mark();
    int64_t pairs = 0;
    TCR_CHECK(tile_pass(rows, cols, sym, T, false, count.as<int32_t>(), nullptr, nullptr, nullptr, &pairs, s, sms,
                        &sink));
    const int e1 = ph.mark();
    TCR_CHECK(off64.alloc_owned(sizeof(int64_t) * (n_rows + 1), s));
    TCR_CHECK(scan_exclusive_i32_to_i64(count.as<int32_t>(), off64.as<int64_t>(), n_rows, s));
    int64_t nnz = 0;
    unsigned long long kept = ~0ull;
    TCR_CUDA(cudaMemcpyAsync(&nnz, off64.as<int64_t>() + n_rows, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    if (sink.cursor)
        TCR_CUDA(cudaMemcpyAsync(&kept, sink.cursor, sizeof(kept), cudaMemcpyDeviceToHost, s));
    TCR_CUDA(cudaStreamSynchronize(s));
    const int e2 = ph.mark();
    TCR_CHECK(out_cols.alloc_owned(sizeof(int32_t) * nnz, s));
    TCR_CHECK(cursor.alloc(sizeof(int32_t) * n_rows, s));
    TCR_CUDA(cudaMemsetAsync(cursor.as<void>(), 0, sizeof(int32_t) * n_rows, s));
    if (nnz > 0) {
        if (sink.cursor && (int64_t)kept <= pcap) {
            int* err = reinterpret_cast<int*>(sink.cursor + 1);
            TCR_CHECK(scatter_pairs(sink.pairs, (int64_t)kept, sym, off64.as<int64_t>(), cursor.as<int32_t>(),
                                    out_cols.as<int32_t>(), err, s));
            int h_err = 0;
            TCR_CUDA(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s));
            TCR_CUDA(cudaStreamSynchronize(s));
            if (h_err) return TCRNET_EDEVICE;
        } else {
            TCR_CHECK(tile_pass(rows, cols, sym, T, true, nullptr, off64.as<int64_t>(), cursor.as<int32_t>(),
                                out_cols.as<int32_t>(), nullptr, s, sms));
        }
    }
    const int e3 = ph.mark();
    TCR_CHECK(sort_rows(off64.as<int64_t>(), out_cols.as<int32_t>(), n_rows, s, sms));
    const int e4 = ph.mark();
    TCR_CHECK(export_csr(h, off64, out_cols, count, n_rows, nnz, force64, s));
    st.candidate_pairs = pairs;
    st.ms_count = ph.ms(e0, e1);
    st.ms_scan = ph.ms(e1, e2);
    st.ms_write = ph.ms(e2, e3);
    st.ms_sort = ph.ms(e3, e4);
    return TCRNET_OK;
}

struct Inputs {
    DevBuf chars, offs;
    const uint8_t* d_chars = nullptr;
    const int64_t* d_offs = nullptr;
    int64_t base = 0;
    int64_t lo = INT64_MIN, hi = INT64_MAX;  // byte offsets the strings must stay in (host inputs)
};

// Device views of flat inputs; host inputs are uploaded on the stream.
tcrnet_status stage_inputs(const uint8_t* chars, const int64_t* offsets, int64_t n, int mem, Inputs& in,
                           cudaStream_t s) {
    if (n == 0) return TCRNET_OK;
    if (!chars || !offsets) return TCRNET_EINVAL;
    if (mem == TCRNET_DEVICE) {
        in.d_chars = chars;
        in.d_offs = offsets;
        in.base = 0;
        return TCRNET_OK;
    }
    if (mem != TCRNET_HOST) return TCRNET_EINVAL;
    // Bytes [offsets[0], offsets[n]) are uploaded; the encoder checks that every
    // string lies inside them (and that offsets do not decrease), per string.
    const int64_t base = offsets[0];
    const int64_t total = offsets[n] - base;
    if (base < 0 || total < 0) return TCRNET_EINVAL;
    TCR_CHECK(in.chars.alloc((size_t)total, s));
    TCR_CHECK(in.offs.alloc(sizeof(int64_t) * (n + 1), s));
    if (total > 0)
        TCR_CUDA(cudaMemcpyAsync(in.chars.as<void>(), chars + base, (size_t)total, cudaMemcpyHostToDevice, s));
    TCR_CUDA(cudaMemcpyAsync(in.offs.as<void>(), offsets, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, s));
    in.d_chars = in.chars.as<uint8_t>();
    in.d_offs = in.offs.as<int64_t>();
    in.base = base;
    in.lo = base;
    in.hi = base + total;
    return TCRNET_OK;
}

// Flatten NUL-terminated host strings.
tcrnet_status flatten(const char* const* seqs, int64_t n, std::vector<uint8_t>& chars, std::vector<int64_t>& offs) {
    if (n > 0 && !seqs) return TCRNET_EINVAL;
    offs.resize((size_t)n + 1);
    offs[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (!seqs[i]) {
            t_last_bad = i;
            return TCRNET_EINVAL;
        }
        offs[i + 1] = offs[i] + (int64_t)std::strlen(seqs[i]);
    }
    chars.resize((size_t)offs[n] + 1);
    for (int64_t i = 0; i < n; ++i) std::memcpy(chars.data() + offs[i], seqs[i], (size_t)(offs[i + 1] - offs[i]));
    return TCRNET_OK;
}

// Largest repertoire the deletion method takes under these options (its join
// records hold 25-bit distinct-string ids; options.deletion_max_n lowers the
// limit for tests).
int64_t deletion_limit(const tcrnet_options& opt) {
    return (opt.deletion_max_n > 0 && opt.deletion_max_n < kDeletionMaxN) ? (int64_t)opt.deletion_max_n
                                                                          : kDeletionMaxN;
}

// The method AUTO stands for: the deletion method from its size cut-over on
// (l_max <= 2) up to its limit, else the all-pairs kernels, which take any n.
int auto_method(int64_t n, int32_t T, int64_t del_limit) {
    if (n > del_limit) return TCRNET_METHOD_TILE;
    if (T <= 1 && n >= kAutoDeletionMinN) return TCRNET_METHOD_DELETION;
    if (T == 2 && n >= kAutoDeletion2MinN) return TCRNET_METHOD_DELETION;
    return TCRNET_METHOD_TILE;
}

// Network of an encoded, bucketed repertoire (pk) into handle h by the method
// the options select: CSR, degree, resident repertoire and, for the deletion
// method, the query index.
tcrnet_status build_from_packed(tcrnet_graph* h, Packed& pk, int64_t n, int32_t T, const tcrnet_options& opt,
                                Phases& ph, cudaStream_t s, int sms, bool keep_index = true) {
    tcrnet_status st = TCRNET_OK;
    int method = opt.method;
    if (method == TCRNET_METHOD_AUTO) method = auto_method(n, T, deletion_limit(opt));
    if (method == TCRNET_METHOD_DELETION && n > deletion_limit(opt)) return TCRNET_ENOTSUP;
    h->stats.method = method;
    for (int L = 0; L < kMaxLen + 2; ++L) h->bucket_off[L] = pk.bucket_off[L];
    if (n == 0) {
        DevBuf off64, cols, deg;
        if ((st = off64.alloc_owned(sizeof(int64_t), s)) != TCRNET_OK) return st;
        if (cudaMemsetAsync(off64.as<void>(), 0, sizeof(int64_t), s) != cudaSuccess) return TCRNET_EDEVICE;
        if ((st = cols.alloc_owned(0, s)) != TCRNET_OK) return st;
        if ((st = deg.alloc_owned(0, s)) != TCRNET_OK) return st;
        if ((st = export_csr(h, off64, cols, deg, 0, 0, opt.force_offsets64 != 0, s)) != TCRNET_OK) return st;
    } else if (method == TCRNET_METHOD_TILE) {
        TileSide side{pk.canon.as<Canon>(), pk.perm.as<int32_t>(), pk.bucket_off};
        st = tile_method(h, side, side, n, true, T, opt.force_offsets64 != 0, ph, s, sms);
        if (st != TCRNET_OK) return st;
    } else {
        DeletionResult dr;
        // (a build with truncated record hashes keeps its index for the
        // analytics, not for queries: they hash their variants in full)
        const int hash_bits = (opt.record_hash_bits > 0 && opt.record_hash_bits < 32) ? opt.record_hash_bits : 32;
        st = deletion_build(pk, T, dr, s, sms, opt.profile != 0, opt.partition_cap, keep_index,
                            opt.partition_target, opt.force_offsets64 != 0, hash_bits);
        if (st != TCRNET_OK) {
            if (dr.bad_index >= 0) t_last_bad = dr.bad_index;  // the encoder's deferred error
            return st;
        }
        h->stats.n_unique = dr.n_unique;
        h->stats.n_records = dr.n_records;
        h->stats.unique_edges = dr.unique_edges;
        h->stats.candidate_pairs = dr.candidates;  // l_max = 2: pairs checked with the exact distance
        h->stats.n_fallback = dr.n_fallback;
        h->stats.closed_total = dr.closed_total;
        h->stats.two_pass_join = dr.two_pass_join;
        h->stats.rejected_candidates = dr.rejected;
        h->stats.ms_count = dr.ms_join;
        h->stats.ms_scan = dr.ms_scan;
        h->stats.ms_write = dr.ms_fill;
        h->stats.ms_sort = dr.ms_sort;
        for (int k = 0; k < 8; ++k) h->stats.ms_phase[k] = dr.ms_phase[k];
        h->ix = dr.index;  // owned by the handle from here on
        dr.index = DeletionIndex();
        st = export_csr(h, dr.off64, dr.cols, dr.degree, n, dr.nnz, opt.force_offsets64 != 0, s, &dr.off32);
        if (st != TCRNET_OK) return st;
    }
    // keep the repertoire resident for queries and inserts: the bucketed copy
    // of a tile build, the input-order copy of a deletion build
    h->lensum = pk.lensum;
    if (pk.canon.as<void>()) {
        h->d_bcanon = static_cast<Canon*>(pk.canon.release());
        h->d_bperm = static_cast<int32_t*>(pk.perm.release());
    } else if (keep_index) {
        h->d_canon_in = static_cast<Canon*>(pk.canon_in.release());
        h->d_lens = static_cast<uint8_t*>(pk.lens.release());
    }
    return TCRNET_OK;
}

tcrnet_status build_impl(const uint8_t* chars, const int64_t* offsets, int64_t n, int mem, int32_t T,
                         const tcrnet_options* opt_in, tcrnet_handle* out, const int64_t* rep_off = nullptr,
                         int64_t nrep = 0) {
    if (!out) return TCRNET_EINVAL;
    *out = nullptr;
    t_last_bad = -1;
    tcrnet_options opt;
    tcrnet_options_init(&opt);
    if (opt_in) opt = *opt_in;
    AllocFaultScope fault_scope(opt.fail_alloc_at);
    if (n < 0 || n > 0x7fffffffLL) return TCRNET_EINVAL;
    if (T < 0) return TCRNET_EINVAL;
    if (opt.method < TCRNET_METHOD_AUTO || opt.method > TCRNET_METHOD_DELETION) return TCRNET_EINVAL;
    if (opt.partition_target != 0 && (opt.partition_target < 4 || opt.partition_target > 128)) return TCRNET_EINVAL;
    if (opt.link_attempts < 0 || opt.deletion_max_n < 0) return TCRNET_EINVAL;
    if (opt.record_hash_bits < 0 || opt.record_hash_bits > 32) return TCRNET_EINVAL;
    if (T > 2 && opt.method == TCRNET_METHOD_DELETION) return TCRNET_ENOTSUP;  // deletion method: l_max <= 2
    if (opt.method == TCRNET_METHOD_DELETION && n > deletion_limit(opt)) return TCRNET_ENOTSUP;
    if (rep_off) {
        // batched: one deletion-method pass over all repertoires
        if (T > 2 || opt.method == TCRNET_METHOD_TILE) return TCRNET_ENOTSUP;
        if (nrep < 1 || nrep > 65536 || rep_off[0] != 0 || rep_off[nrep] != n) return TCRNET_EINVAL;
        for (int64_t r = 0; r < nrep; ++r)
            if (rep_off[r + 1] < rep_off[r]) return TCRNET_EINVAL;
        if (n > deletion_limit(opt)) return TCRNET_ENOTSUP;  // one deletion pass over all repertoires
        opt.method = TCRNET_METHOD_DELETION;
    }
    if (opt.method == TCRNET_METHOD_AUTO)  // decided before packing: only the tile method buckets
        opt.method = auto_method(n, T, deletion_limit(opt));
    DeviceGuard dg;
    TCR_CHECK(dg.set(opt.device));
    int dev = 0;
    TCR_CUDA(cudaGetDevice(&dev));
    configure_pool(dev);
    cudaStream_t s = (cudaStream_t)opt.stream;
    const int sms = sm_count(dev);

    tcrnet_graph* h = new (std::nothrow) tcrnet_graph();
    if (!h) return TCRNET_ENOMEM;
    std::memset(&h->stats, 0, sizeof(h->stats));
    h->device = dev;
    h->stream = s;
    h->threshold = T;
    h->stats.threshold = T;
    h->stats.n = n;

    ArenaLease lease(dev, s);
    Phases ph(opt.profile != 0, s);
    const int64_t launches0 = launches_so_far();
    auto fail = [&](tcrnet_status st) {
        cudaStreamSynchronize(s);
        free_handle_memory(h);
        delete h;
        return st;
    };
    const int p0 = ph.mark();
    Inputs in;
    tcrnet_status st = stage_inputs(chars, offsets, n, mem, in, s);
    if (st != TCRNET_OK) return fail(st);
    const int p1 = ph.mark();
    Packed pk;
    int64_t bad = -1;
    if (n > 0) {
        // A deletion build at l_max <= 1 does not wait for the encoder: the
        // total length (which sizes its records) is the byte span of the
        // strings, offsets[n] - offsets[0], exact for valid input, and the
        // encoder's error word is checked at the build's first readback. The
        // span is read before the encoder runs (host inputs: on the host).
        int64_t span = -1;
        cudaEvent_t span_ready = nullptr;
        int64_t* pin = static_cast<int64_t*>(pinned_scratch());
        const bool defer = opt.method == TCRNET_METHOD_DELETION && T <= 1 && !rep_off && pin;
        if (defer && mem == TCRNET_HOST) {
            span = offsets[n] - offsets[0];
        } else if (defer) {
            TCR_CUDA(cudaMemcpyAsync(pin, in.d_offs, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            TCR_CUDA(cudaMemcpyAsync(pin + 1, in.d_offs + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            span_ready = event_acquire();
            if (span_ready) TCR_CUDA(cudaEventRecord(span_ready, s));
        }
        // chars are addressed as d_chars + (offsets[i] - base)
        st = pack_strings(in.d_chars - in.base, in.d_offs, n, pk, &bad, s, opt.method == TCRNET_METHOD_TILE,
                          opt.method != TCRNET_METHOD_TILE && !rep_off, in.lo, in.hi, defer);
        if (defer && mem != TCRNET_HOST) {
            if (span_ready) {
                const cudaError_t e = cudaEventSynchronize(span_ready);
                event_release(span_ready);
                if (e != cudaSuccess) return fail(TCRNET_EDEVICE);
            } else if (cudaStreamSynchronize(s) != cudaSuccess) {
                return fail(TCRNET_EDEVICE);
            }
            span = pin[1] - pin[0];
        }
        if (st != TCRNET_OK) {
            t_last_bad = bad;
            return fail(st);
        }
        if (defer) {
            if (span >= n && span <= (int64_t)kMaxLen * n) {
                pk.lensum = span;
            } else {  // not a valid input: the encoder has flagged it; report its error now
                unsigned long long fl[2] = {0, 0};
                if (cudaMemcpyAsync(fl, pk.flags.as<void>(), sizeof(fl), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                    cudaStreamSynchronize(s) != cudaSuccess)
                    return fail(TCRNET_EDEVICE);
                st = pack_flags_status(fl[0], &bad);
                if (st != TCRNET_OK) {
                    t_last_bad = bad;
                    return fail(st);
                }
                pk.lensum = (int64_t)fl[1];
            }
        }
    }
    if (rep_off && n > 0) {
        st = tag_repertoires(pk.canon_in.as<Canon>(), n, rep_off, nrep, s);
        if (st != TCRNET_OK) return fail(st);
        h->batched = true;
    }
    const int p2 = ph.mark();
    st = build_from_packed(h, pk, n, T, opt, ph, s, sms, /*keep_index=*/rep_off == nullptr);
    if (st != TCRNET_OK) return fail(st);
    const int p3 = ph.mark();
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(TCRNET_EDEVICE);
    h->stats.nnz = h->nnz;
    h->stats.kernel_launches = launches_so_far() - launches0;
    h->stats.ms_upload = ph.ms(p0, p1);
    h->stats.ms_pack = ph.ms(p1, p2);
    h->stats.ms_total = ph.ms(p0, p3);
    *out = h;
    return TCRNET_OK;
}

}  // namespace
}  // namespace tcr

using namespace tcr;

extern "C" {

void tcrnet_options_init(tcrnet_options* opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->method = TCRNET_METHOD_AUTO;
    opt->device = -1;
}

tcrnet_status tcrnet_build_flat(const uint8_t* chars, const int64_t* offsets, int64_t n, int32_t mem,
                                int32_t threshold, const tcrnet_options* opt, tcrnet_handle* out) {
    return build_impl(chars, offsets, n, mem, threshold, opt, out);
}

tcrnet_status tcrnet_build_batched(const uint8_t* chars, const int64_t* offsets, int64_t n,
                                   const int64_t* rep_offsets, int64_t nrep, int32_t mem, int32_t threshold,
                                   const tcrnet_options* opt, tcrnet_handle* out) {
    if (!rep_offsets) return TCRNET_EINVAL;
    return build_impl(chars, offsets, n, mem, threshold, opt, out, rep_offsets, nrep);
}

tcrnet_status tcrnet_build(const char* const* seqs, int64_t n, int32_t threshold, const tcrnet_options* opt,
                           tcrnet_handle* out) {
    if (out) *out = nullptr;
    t_last_bad = -1;
    if (n < 0) return TCRNET_EINVAL;
    std::vector<uint8_t> chars;
    std::vector<int64_t> offs;
    TCR_CHECK(flatten(seqs, n, chars, offs));
    return build_impl(chars.data(), offs.data(), n, TCRNET_HOST, threshold, opt, out);
}

tcrnet_status tcrnet_info(tcrnet_handle h, int64_t* n, int64_t* nnz, int32_t* off64) {
    if (!h) return TCRNET_EINVAL;
    if (n) *n = h->n;
    if (nnz) *nnz = h->nnz;
    if (off64) *off64 = h->offsets64;
    return TCRNET_OK;
}

tcrnet_status tcrnet_copy_csr(tcrnet_handle h, void* offsets, int32_t* cols, int32_t* degree, int32_t mem) {
    if (!h) return TCRNET_EINVAL;
    if (mem != TCRNET_HOST && mem != TCRNET_DEVICE) return TCRNET_EINVAL;
    DeviceGuard dg;
    TCR_CHECK(dg.set(h->device));
    const cudaMemcpyKind kind = mem == TCRNET_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    cudaStream_t s = h->stream;
    if (offsets)
        TCR_CUDA(cudaMemcpyAsync(offsets, h->d_offsets, (h->offsets64 ? 8 : 4) * (size_t)(h->n + 1), kind, s));
    if (cols && h->nnz > 0) TCR_CUDA(cudaMemcpyAsync(cols, h->d_cols, sizeof(int32_t) * (size_t)h->nnz, kind, s));
    if (degree && h->n > 0) TCR_CUDA(cudaMemcpyAsync(degree, h->d_degree, sizeof(int32_t) * (size_t)h->n, kind, s));
    TCR_CUDA(cudaStreamSynchronize(s));
    return TCRNET_OK;
}

tcrnet_status tcrnet_csr_device(tcrnet_handle h, const void** offsets, const int32_t** cols, const int32_t** degree) {
    if (!h) return TCRNET_EINVAL;
    if (offsets) *offsets = h->d_offsets;
    if (cols) *cols = h->d_cols;
    if (degree) *degree = h->d_degree;
    return TCRNET_OK;
}

tcrnet_status tcrnet_query_ex(tcrnet_handle h, const uint8_t* chars, const int64_t* offsets, int64_t m, int32_t mem,
                              const tcrnet_options* opt, tcrnet_handle* out) {
    if (!out) return TCRNET_EINVAL;
    *out = nullptr;
    t_last_bad = -1;
    if (!h || m < 0 || m > 0x7fffffffLL) return TCRNET_EINVAL;
    if (h->query_result || h->batched) return TCRNET_ESTATE;
    int method = opt ? opt->method : TCRNET_METHOD_AUTO;
    if (method < TCRNET_METHOD_AUTO || method > TCRNET_METHOD_DELETION) return TCRNET_EINVAL;
    if (method == TCRNET_METHOD_AUTO) method = h->ix.valid() ? TCRNET_METHOD_DELETION : TCRNET_METHOD_TILE;
    if (method == TCRNET_METHOD_DELETION && !h->ix.valid()) return TCRNET_ENOTSUP;
    AllocFaultScope fault_scope(opt ? opt->fail_alloc_at : 0);
    DeviceGuard dg;
    TCR_CHECK(dg.set(h->device));
    cudaStream_t s = (opt && opt->stream) ? (cudaStream_t)opt->stream : h->stream;
    const int sms = sm_count(h->device);
    tcrnet_graph* r = new (std::nothrow) tcrnet_graph();
    if (!r) return TCRNET_ENOMEM;
    std::memset(&r->stats, 0, sizeof(r->stats));
    r->device = h->device;
    r->stream = s;
    r->query_result = true;
    r->threshold = h->threshold;
    r->stats.threshold = h->threshold;
    r->stats.n = m;
    r->stats.method = method;
    auto fail = [&](tcrnet_status st) {
        cudaStreamSynchronize(s);
        free_handle_memory(r);
        delete r;
        return st;
    };
    ArenaLease lease(h->device, s);
    Phases ph(false, s);
    const int64_t launches0 = launches_so_far();
    Inputs in;
    tcrnet_status st = stage_inputs(chars, offsets, m, mem, in, s);
    if (st != TCRNET_OK) return fail(st);
    if (m == 0) {
        DevBuf off64, cols, deg;
        if ((st = off64.alloc_owned(sizeof(int64_t), s)) != TCRNET_OK) return fail(st);
        if (cudaMemsetAsync(off64.as<void>(), 0, sizeof(int64_t), s) != cudaSuccess) return fail(TCRNET_EDEVICE);
        if ((st = cols.alloc_owned(0, s)) != TCRNET_OK) return fail(st);
        if ((st = deg.alloc_owned(0, s)) != TCRNET_OK) return fail(st);
        if ((st = export_csr(r, off64, cols, deg, 0, 0, false, s)) != TCRNET_OK) return fail(st);
    } else {
        Packed pk;
        int64_t bad = -1;
        st = pack_strings(in.d_chars - in.base, in.d_offs, m, pk, &bad, s, method != TCRNET_METHOD_DELETION, false,
                          in.lo, in.hi);
        if (st != TCRNET_OK) {
            t_last_bad = bad;
            return fail(st);
        }
        if (method == TCRNET_METHOD_DELETION) {
            DevBuf off64, cols, cnt;
            int64_t nnz = 0;
            st = deletion_query(h->ix, pk, h->threshold, off64, cols, cnt, &nnz, s, sms);
            if (st != TCRNET_OK) return fail(st);
            st = export_csr(r, off64, cols, cnt, m, nnz, false, s);
            if (st != TCRNET_OK) return fail(st);
        } else {
            TileSide qs{pk.canon.as<Canon>(), pk.perm.as<int32_t>(), pk.bucket_off};
            TileSide rs{h->d_bcanon, h->d_bperm, h->bucket_off};
            Packed rb;  // a deletion build keeps its strings in input order: bucket them for this call
            if (!h->d_bcanon && h->n > 0) {
                st = bucket_from(h->d_canon_in, h->d_lens, h->n, rb, s);
                if (st != TCRNET_OK) return fail(st);
                rs = TileSide{rb.canon.as<Canon>(), rb.perm.as<int32_t>(), rb.bucket_off};
            }
            st = tile_method(r, qs, rs, m, false, h->threshold, false, ph, s, sms);
            if (st != TCRNET_OK) return fail(st);
        }
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(TCRNET_EDEVICE);
    r->stats.nnz = r->nnz;
    r->stats.kernel_launches = launches_so_far() - launches0;
    *out = r;
    return TCRNET_OK;
}

tcrnet_status tcrnet_query_flat(tcrnet_handle h, const uint8_t* chars, const int64_t* offsets, int64_t m,
                                int32_t mem, tcrnet_handle* out) {
    return tcrnet_query_ex(h, chars, offsets, m, mem, nullptr, out);
}

tcrnet_status tcrnet_query(tcrnet_handle h, const char* const* queries, int64_t m, tcrnet_handle* out) {
    if (out) *out = nullptr;
    t_last_bad = -1;
    if (m < 0) return TCRNET_EINVAL;
    std::vector<uint8_t> chars;
    std::vector<int64_t> offs;
    TCR_CHECK(flatten(queries, m, chars, offs));
    return tcrnet_query_flat(h, chars.data(), offs.data(), m, TCRNET_HOST, out);
}

}  // extern "C"

namespace tcr {
namespace {

// Largest mean records per partition that a merged insert may leave behind
// (builds aim at 24 or 32).
constexpr int64_t kMergeMaxPartitionFill = 48;
// A merge copies the whole network and index once, queries the new strings
// and runs about 60 small steps (~0.5 ms whatever the size); a rebuild grows
// faster than linearly with the repertoire. Measured on a B300 (synthetic
// repertoires, l_max = 1, copy-on-write inserts): rebuilds win below ~7e5
// resident strings (3e5: 0.39 against 0.59 ms), merges of a few hundred
// strings win from there (8e5: 100 new strings 0.78 against 0.80 ms, 1,000
// new strings 0.83 against 0.82 ms), and from 1.5e6 merges of up to 1/32 (2e6
// and 62,500 new strings: 1.94 against 2.80 ms).
bool merge_is_faster(int64_t n_old, int64_t m) {
    if (n_old >= 1500000) return m * 32 <= n_old;
    if (n_old >= 700000) return m * 2048 <= n_old;
    return false;
}

// The network of h's strings followed by m new ones, as a new graph; h is only
// read (its resident strings, network and index), so queries on h may run
// meanwhile on other streams.
tcrnet_status extend_impl(tcrnet_handle h, const uint8_t* chars, const int64_t* offsets, int64_t m, int32_t mem,
                          const tcrnet_options* opt_in, tcrnet_graph** out) {
    *out = nullptr;
    const int64_t n_old = h->n;
    const int64_t N = n_old + m;
    if (N > 0x7fffffffLL) return TCRNET_EINVAL;
    tcrnet_options opt;
    tcrnet_options_init(&opt);
    opt.method = h->stats.method;  // the grown repertoire is built the way the handle was
    opt.force_offsets64 = (h->offsets64 && h->nnz <= 0x7fffffffLL) ? 1 : 0;
    if (opt_in) {
        opt.stream = opt_in->stream;
        opt.profile = opt_in->profile;
        opt.fail_alloc_at = opt_in->fail_alloc_at;
        opt.insert_rebuild = opt_in->insert_rebuild;
        if (opt.insert_rebuild < 0 || opt.insert_rebuild > 2) return TCRNET_EINVAL;
        opt.deletion_max_n = opt_in->deletion_max_n;
        if (opt.deletion_max_n < 0) return TCRNET_EINVAL;
    }
    // past the deletion method's limit the grown repertoire is built by the
    // tile method (the method AUTO would take)
    if (opt.method == TCRNET_METHOD_DELETION && N > deletion_limit(opt)) opt.method = TCRNET_METHOD_TILE;
    AllocFaultScope fault_scope(opt.fail_alloc_at);
    DeviceGuard dg;
    TCR_CHECK(dg.set(h->device));
    cudaStream_t s = opt.stream ? (cudaStream_t)opt.stream : h->stream;
    opt.stream = s;
    const int sms = sm_count(h->device);
    ArenaLease lease(h->device, s);
    Phases ph(opt.profile != 0, s);
    const int64_t launches0 = launches_so_far();
    Inputs in;
    TCR_CHECK(stage_inputs(chars, offsets, m, mem, in, s));
    Packed pn;
    int64_t bad = -1;
    tcrnet_status st = pack_strings(in.d_chars - in.base, in.d_offs, m, pn, &bad, s, /*bucket=*/false, false, in.lo,
                                    in.hi);
    if (st != TCRNET_OK) {
        t_last_bad = bad;
        return st;
    }
    // the grown repertoire: resident strings (input order) then the new ones;
    // a deletion rebuild keeps this input-order copy, a tile rebuild buckets it
    const bool tile = opt.method == TCRNET_METHOD_TILE;
    Packed pk;
    pk.n = N;
    pk.lensum = h->lensum + pn.lensum;
    if (tile) {
        TCR_CHECK(pk.canon_in.alloc(sizeof(Canon) * N, s));
        TCR_CHECK(pk.lens.alloc(N, s));
    } else {
        TCR_CHECK(pk.canon_in.alloc_owned(sizeof(Canon) * N, s));
        TCR_CHECK(pk.lens.alloc_owned(N, s));
    }
    if (h->d_canon_in) {
        if (n_old > 0) {
            TCR_CUDA(cudaMemcpyAsync(pk.canon_in.as<Canon>(), h->d_canon_in, sizeof(Canon) * n_old,
                                     cudaMemcpyDeviceToDevice, s));
            TCR_CUDA(cudaMemcpyAsync(pk.lens.as<uint8_t>(), h->d_lens, n_old, cudaMemcpyDeviceToDevice, s));
        }
    } else {
        TCR_CHECK(unbucket_strings(h->d_bcanon, h->d_bperm, h->bucket_off, n_old, pk.canon_in.as<Canon>(),
                                   pk.lens.as<uint8_t>(), s));
    }
    if (m > 0) {
        TCR_CUDA(cudaMemcpyAsync(pk.canon_in.as<Canon>() + n_old, pn.canon_in.as<Canon>(), sizeof(Canon) * m,
                                 cudaMemcpyDeviceToDevice, s));
        TCR_CUDA(cudaMemcpyAsync(pk.lens.as<uint8_t>() + n_old, pn.lens.as<uint8_t>(), m,
                                 cudaMemcpyDeviceToDevice, s));
    }
    if (tile) TCR_CHECK(bucket_strings(pk, s));
    // A deletion build's network and index can take the new strings without a
    // rebuild, while its partitions stay small (they were sized for the
    // original record count; a rebuild re-sizes them) and the insert is small
    // next to the repertoire.
    const DeletionIndex& ix = h->ix;
    const bool can_merge = !tile && opt.insert_rebuild != 1 && m > 0 && ix.valid() && ix.uid && ix.n == n_old &&
                           h->threshold == 1 && N <= deletion_limit(opt) &&
                           ix.R + m + pn.lensum <= kMergeMaxPartitionFill * ix.P;
    const bool merge = can_merge && (opt.insert_rebuild == 2 || merge_is_faster(n_old, m));
    tcrnet_graph* g = new (std::nothrow) tcrnet_graph();
    if (!g) return TCRNET_ENOMEM;
    std::memset(&g->stats, 0, sizeof(g->stats));
    g->device = h->device;
    g->stream = h->stream;
    g->threshold = h->threshold;
    g->stats.threshold = h->threshold;
    g->stats.n = N;
    if (merge) {
        CsrView gv;
        gv.offsets = h->d_offsets;
        gv.off64 = h->offsets64 != 0;
        gv.cols = h->d_cols;
        gv.degree = h->d_degree;
        gv.n = n_old;
        gv.nnz = h->nnz;
        InsertResult ir;
        st = deletion_insert(ix, gv, pn, h->threshold, ir, s, sms, opt.profile != 0);
        if (st == TCRNET_OK) {
            g->ix = ir.index;  // owned by g from here on (freed with it on a later error)
            ir.index = DeletionIndex();
            g->stats.method = TCRNET_METHOD_DELETION;
            g->stats.n_unique = g->ix.U;
            g->stats.n_records = g->ix.R;
            g->stats.unique_edges = g->ix.E;
            g->stats.merged_inserts = h->stats.merged_inserts + 1;
            for (int k = 0; k < 8; ++k) g->stats.ms_phase[k] = ir.ms_phase[k];
            g->stats.ms_total = ir.ms_phase[7];
            st = export_csr(g, ir.off64, ir.cols, ir.degree, N, ir.nnz, opt.force_offsets64 != 0, s);
        }
        if (st == TCRNET_OK) {
            g->lensum = pk.lensum;
            g->d_canon_in = static_cast<Canon*>(pk.canon_in.release());
            g->d_lens = static_cast<uint8_t*>(pk.lens.release());
        }
    } else {
        st = build_from_packed(g, pk, N, h->threshold, opt, ph, s, sms);
    }
    if (st == TCRNET_OK && cudaStreamSynchronize(s) != cudaSuccess) st = TCRNET_EDEVICE;
    if (st != TCRNET_OK) {
        cudaStreamSynchronize(s);
        free_handle_memory(g);
        delete g;
        return st;  // the handle keeps its previous network
    }
    g->stats.nnz = g->nnz;
    g->stats.kernel_launches = launches_so_far() - launches0;
    *out = g;
    return TCRNET_OK;
}

}  // namespace
}  // namespace tcr

extern "C" {

tcrnet_status tcrnet_insert_ex(tcrnet_handle h, const uint8_t* chars, const int64_t* offsets, int64_t m, int32_t mem,
                               const tcrnet_options* opt_in) {
    t_last_bad = -1;
    if (!h || m < 0) return TCRNET_EINVAL;
    if (h->query_result || h->batched) return TCRNET_ESTATE;
    if (m == 0) return TCRNET_OK;
    tcrnet_graph* g = nullptr;
    const tcrnet_status st = extend_impl(h, chars, offsets, m, mem, opt_in, &g);
    if (st != TCRNET_OK) return st;  // the handle keeps its previous network
    {
        DeviceGuard dg;
        TCR_CHECK(dg.set(h->device));
        free_handle_memory(h);
    }
    *h = *g;  // plain pointers and sizes: the handle now owns g's memory
    delete g;
    return TCRNET_OK;
}

tcrnet_status tcrnet_extend(tcrnet_handle h, const uint8_t* chars, const int64_t* offsets, int64_t m, int32_t mem,
                            const tcrnet_options* opt, tcrnet_handle* out) {
    t_last_bad = -1;
    if (!out) return TCRNET_EINVAL;
    *out = nullptr;
    if (!h || m < 0) return TCRNET_EINVAL;
    if (h->query_result || h->batched) return TCRNET_ESTATE;
    tcrnet_graph* g = nullptr;  // m == 0: a rebuilt copy, a handle of its own
    const tcrnet_status st = extend_impl(h, chars, offsets, m, mem, opt, &g);
    if (st != TCRNET_OK) return st;
    *out = g;
    return TCRNET_OK;
}

tcrnet_status tcrnet_insert_flat(tcrnet_handle h, const uint8_t* chars, const int64_t* offsets, int64_t m,
                                 int32_t mem) {
    return tcrnet_insert_ex(h, chars, offsets, m, mem, nullptr);
}

tcrnet_status tcrnet_insert(tcrnet_handle h, const char* const* seqs, int64_t m) {
    t_last_bad = -1;
    if (m < 0) return TCRNET_EINVAL;
    std::vector<uint8_t> chars;
    std::vector<int64_t> offs;
    TCR_CHECK(flatten(seqs, m, chars, offs));
    return tcrnet_insert_ex(h, chars.data(), offs.data(), m, TCRNET_HOST, nullptr);
}

tcrnet_status tcrnet_sort_rows(const int64_t* d_offsets, int32_t* d_cols, int64_t n, void* stream) {
    t_last_bad = -1;
    if (n < 0 || (n > 0 && (!d_offsets || !d_cols))) return TCRNET_EINVAL;
    if (n == 0) return TCRNET_OK;
    int dev = 0;
    TCR_CUDA(cudaGetDevice(&dev));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    {
        ArenaLease lease(dev, s);
        TCR_CHECK(tcr::sort_rows(d_offsets, d_cols, n, s, sm_count(dev)));
    }
    TCR_CUDA(cudaStreamSynchronize(s));
    return TCRNET_OK;
}

tcrnet_status tcrnet_components(tcrnet_handle h, const uint8_t* keep, int32_t* labels, int32_t mem,
                                int64_t* n_components, int64_t* largest) {
    return tcrnet_components_ex(h, keep, labels, mem, nullptr, n_components, largest);
}

tcrnet_status tcrnet_components_ex(tcrnet_handle h, const uint8_t* keep, int32_t* labels, int32_t mem,
                                   const tcrnet_options* opt, int64_t* n_components, int64_t* largest) {
    if (n_components) *n_components = 0;
    if (largest) *largest = 0;
    if (!h || (mem != TCRNET_HOST && mem != TCRNET_DEVICE)) return TCRNET_EINVAL;
    if (opt && opt->link_attempts < 0) return TCRNET_EINVAL;
    const int attempts = opt ? opt->link_attempts : 0;
    DeviceGuard dg;
    TCR_CHECK(dg.set(h->device));
    cudaStream_t s = (opt && opt->stream) ? (cudaStream_t)opt->stream : h->stream;
    const int64_t n = h->n;
    int64_t nc = 0, lc = 0;
    if (n > 0) {
        ArenaLease lease(h->device, s);
        DevBuf dkeep, dlab;
        const uint8_t* k = keep;
        int32_t* lab = labels;
        if (mem == TCRNET_HOST) {
            if (keep) {
                TCR_CHECK(dkeep.alloc(n, s));
                TCR_CUDA(cudaMemcpyAsync(dkeep.as<void>(), keep, n, cudaMemcpyHostToDevice, s));
                k = dkeep.as<uint8_t>();
            }
            TCR_CHECK(dlab.alloc(sizeof(int32_t) * n, s));
            lab = dlab.as<int32_t>();
        } else if (!lab) {
            TCR_CHECK(dlab.alloc(sizeof(int32_t) * n, s));
            lab = dlab.as<int32_t>();
        }
        if (h->ix.uid) {  // a deletion build: the graph of distinct strings gives the same components
            TCR_CHECK(components_distinct(h->ix.uid, n, h->ix.uedges, h->ix.E, h->ix.U, k, labels ? lab : nullptr, &nc,
                                          &lc, s, sm_count(h->device), attempts));
        } else {
            TCR_CHECK(components(h->d_offsets, h->offsets64 != 0, h->d_cols, n, k, lab, &nc, &lc, s,
                                 sm_count(h->device), attempts));
        }
        if (mem == TCRNET_HOST && labels)
            TCR_CUDA(cudaMemcpyAsync(labels, lab, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
        TCR_CUDA(cudaStreamSynchronize(s));
    }
    if (n_components) *n_components = nc;
    if (largest) *largest = lc;
    return TCRNET_OK;
}

tcrnet_status tcrnet_neighbor_degree(tcrnet_handle h, double* knn, int32_t mem) {
    if (!h || !knn || (mem != TCRNET_HOST && mem != TCRNET_DEVICE)) return TCRNET_EINVAL;
    DeviceGuard dg;
    TCR_CHECK(dg.set(h->device));
    cudaStream_t s = h->stream;
    const int64_t n = h->n;
    if (n == 0) return TCRNET_OK;
    ArenaLease lease(h->device, s);
    DevBuf dk;
    double* out = knn;
    if (mem == TCRNET_HOST) {
        TCR_CHECK(dk.alloc(sizeof(double) * n, s));
        out = dk.as<double>();
    }
    if (h->ix.uid) {
        TCR_CHECK(neighbor_degree_distinct(h->ix.uid, n, h->ix.uedges, h->ix.E, h->ix.umult, h->ix.U, out, s,
                                           sm_count(h->device)));
    } else {
        TCR_CHECK(neighbor_degree(h->d_offsets, h->offsets64 != 0, h->d_cols, n, out, s, sm_count(h->device)));
    }
    if (mem == TCRNET_HOST) TCR_CUDA(cudaMemcpyAsync(knn, out, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    TCR_CUDA(cudaStreamSynchronize(s));
    return TCRNET_OK;
}

tcrnet_status tcrnet_degree_histogram(tcrnet_handle h, int64_t* hist, int64_t nbins, int32_t mem,
                                      int64_t* max_degree) {
    if (!h || !hist || nbins < 1 || (mem != TCRNET_HOST && mem != TCRNET_DEVICE)) return TCRNET_EINVAL;
    DeviceGuard dg;
    TCR_CHECK(dg.set(h->device));
    cudaStream_t s = h->stream;
    ArenaLease lease(h->device, s);
    DevBuf dh;
    int64_t* out = hist;
    if (mem == TCRNET_HOST) {
        TCR_CHECK(dh.alloc(sizeof(int64_t) * nbins, s));
        out = dh.as<int64_t>();
    }
    TCR_CHECK(degree_histogram(h->d_degree, h->n, out, nbins, max_degree, s, sm_count(h->device)));
    if (mem == TCRNET_HOST) {
        TCR_CUDA(cudaMemcpyAsync(hist, out, sizeof(int64_t) * nbins, cudaMemcpyDeviceToHost, s));
        TCR_CUDA(cudaStreamSynchronize(s));
    }
    return TCRNET_OK;
}

}  // extern "C"

namespace tcr {
namespace {

// ---- checkpoint file -------------------------------------------------------
// Header (fixed layout, host byte order) then the device arrays, each as a u64
// byte count followed by the bytes. Arrays: offsets, cols, degree, then the
// resident strings (bucketed copy + order, or input-order copy + lengths),
// then the deletion index when present.
constexpr char kMagic[8] = {'T', 'C', 'R', 'N', 'E', 'T', 'C', 'K'};
constexpr uint32_t kFileVersion = 4;

struct FileHeader {
    char magic[8];
    uint32_t version;
    uint32_t header_bytes;
    int32_t threshold, offsets64, batched, has_bucketed, has_input_order, has_index;
    int64_t n, nnz, lensum, ix_U, ix_P, ix_R, ix_E;
    int64_t bucket_off[kMaxLen + 2];
    tcrnet_stats stats;
};

bool write_array(std::FILE* f, const void* dev, uint64_t bytes, cudaStream_t s, std::vector<char>& staging) {
    if (std::fwrite(&bytes, sizeof(bytes), 1, f) != 1) return false;
    if (bytes == 0) return true;
    staging.resize(bytes);
    if (cudaMemcpyAsync(staging.data(), dev, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess) return false;
    if (cudaStreamSynchronize(s) != cudaSuccess) return false;
    return std::fwrite(staging.data(), 1, bytes, f) == bytes;
}

tcrnet_status read_array(std::FILE* f, uint64_t expect, void** dev, cudaStream_t s, std::vector<char>& staging) {
    uint64_t bytes = 0;
    if (std::fread(&bytes, sizeof(bytes), 1, f) != 1 || bytes != expect) return TCRNET_EINVAL;
    DevBuf b;
    TCR_CHECK(b.alloc_owned(bytes, s));
    if (bytes > 0) {
        staging.resize(bytes);
        if (std::fread(staging.data(), 1, bytes, f) != bytes) return TCRNET_EINVAL;
        TCR_CUDA(cudaMemcpyAsync(b.as<void>(), staging.data(), bytes, cudaMemcpyHostToDevice, s));
        TCR_CUDA(cudaStreamSynchronize(s));
    }
    *dev = b.release();
    return TCRNET_OK;
}

}  // namespace
}  // namespace tcr

extern "C" {

tcrnet_status tcrnet_save(tcrnet_handle h, const char* path) {
    if (!h || !path) return TCRNET_EINVAL;
    if (h->query_result) return TCRNET_ESTATE;
    DeviceGuard dg;
    TCR_CHECK(dg.set(h->device));
    FileHeader hd;
    std::memset(&hd, 0, sizeof(hd));
    std::memcpy(hd.magic, kMagic, sizeof(kMagic));
    hd.version = kFileVersion;
    hd.header_bytes = (uint32_t)sizeof(FileHeader);
    hd.threshold = h->threshold;
    hd.offsets64 = h->offsets64;
    hd.batched = h->batched ? 1 : 0;
    hd.has_bucketed = h->d_bcanon ? 1 : 0;
    hd.has_input_order = h->d_canon_in ? 1 : 0;
    hd.has_index = h->ix.valid() ? 1 : 0;
    hd.n = h->n;
    hd.nnz = h->nnz;
    hd.lensum = h->lensum;
    for (int L = 0; L < kMaxLen + 2; ++L) hd.bucket_off[L] = h->bucket_off[L];
    hd.stats = h->stats;
    cudaStream_t s = h->stream;
    if (hd.has_index) {
        hd.ix_U = h->ix.U;
        hd.ix_P = h->ix.P;
        hd.ix_E = h->ix.uid ? h->ix.E : -1;
        TCR_CUDA(cudaMemcpyAsync(&hd.ix_R, h->ix.poff + h->ix.P, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        TCR_CUDA(cudaStreamSynchronize(s));
    }
    std::FILE* f = std::fopen(path, "wb");
    if (!f) return TCRNET_EINVAL;
    std::vector<char> st;
    const uint64_t n = (uint64_t)h->n;
    bool ok = std::fwrite(&hd, sizeof(hd), 1, f) == 1;
    ok = ok && write_array(f, h->d_offsets, (n + 1) * (h->offsets64 ? 8 : 4), s, st);
    ok = ok && write_array(f, h->d_cols, (uint64_t)h->nnz * 4, s, st);
    ok = ok && write_array(f, h->d_degree, n * 4, s, st);
    if (hd.has_bucketed) {
        ok = ok && write_array(f, h->d_bcanon, n * sizeof(Canon), s, st);
        ok = ok && write_array(f, h->d_bperm, n * 4, s, st);
    }
    if (hd.has_input_order) {
        ok = ok && write_array(f, h->d_canon_in, n * sizeof(Canon), s, st);
        ok = ok && write_array(f, h->d_lens, n, s, st);
    }
    if (hd.has_index) {
        ok = ok && write_array(f, h->ix.ucanon, (uint64_t)h->ix.U * sizeof(Canon), s, st);
        ok = ok && write_array(f, h->ix.umult, n * 4, s, st);
        ok = ok && write_array(f, h->ix.mem_off, (n + 1) * 8, s, st);
        ok = ok && write_array(f, h->ix.members, n * 4, s, st);
        ok = ok && write_array(f, h->ix.recs, (uint64_t)hd.ix_R * 8, s, st);
        ok = ok && write_array(f, h->ix.poff, ((uint64_t)h->ix.P + 1) * 8, s, st);
        if (hd.ix_E >= 0) {
            ok = ok && write_array(f, h->ix.uid, n * 4, s, st);
            ok = ok && write_array(f, h->ix.uedges, (uint64_t)hd.ix_E * 8, s, st);
        }
    }
    ok = (std::fclose(f) == 0) && ok;
    return ok ? TCRNET_OK : TCRNET_EINVAL;
}

tcrnet_status tcrnet_load(const char* path, const tcrnet_options* opt_in, tcrnet_handle* out) {
    if (!out) return TCRNET_EINVAL;
    *out = nullptr;
    if (!path) return TCRNET_EINVAL;
    tcrnet_options opt;
    tcrnet_options_init(&opt);
    if (opt_in) opt = *opt_in;
    std::FILE* f = std::fopen(path, "rb");
    if (!f) return TCRNET_EINVAL;
    FileHeader hd;
    // the header is checked before any device work
    const bool head_ok = std::fread(&hd, sizeof(hd), 1, f) == 1 && std::memcmp(hd.magic, kMagic, 8) == 0 &&
                         hd.version == kFileVersion && hd.header_bytes == sizeof(FileHeader) && hd.n >= 0 &&
                         hd.n <= 0x7fffffffLL && hd.nnz >= 0 && hd.threshold >= 0 &&
                         (hd.offsets64 == 0 || hd.offsets64 == 1) && (hd.has_index == 0 || hd.has_index == 1) &&
                         hd.ix_U >= 0 && hd.ix_U <= hd.n && hd.ix_P >= 0 && hd.ix_R >= 0 && hd.ix_E >= -1 &&
                         (hd.offsets64 || hd.nnz <= 0x7fffffffLL);
    if (!head_ok) {
        std::fclose(f);
        return TCRNET_EINVAL;
    }
    DeviceGuard dg;
    tcrnet_status st = dg.set(opt.device);
    if (st != TCRNET_OK) {
        std::fclose(f);
        return st;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    configure_pool(dev);
    cudaStream_t s = (cudaStream_t)opt.stream;
    tcrnet_graph* h = new (std::nothrow) tcrnet_graph();
    if (!h) {
        std::fclose(f);
        return TCRNET_ENOMEM;
    }
    h->device = dev;
    h->stream = s;
    h->threshold = hd.threshold;
    h->batched = hd.batched != 0;
    h->n = hd.n;
    h->nnz = hd.nnz;
    h->offsets64 = hd.offsets64;
    h->lensum = hd.lensum;
    for (int L = 0; L < kMaxLen + 2; ++L) h->bucket_off[L] = hd.bucket_off[L];
    h->stats = hd.stats;
    const uint64_t n = (uint64_t)hd.n;
    std::vector<char> buf;
    void* p = nullptr;
    auto rd = [&](uint64_t bytes) {
        p = nullptr;
        return st == TCRNET_OK ? (st = read_array(f, bytes, &p, s, buf)) : st;
    };
    if (rd((n + 1) * (hd.offsets64 ? 8 : 4)) == TCRNET_OK) h->d_offsets = p;
    if (rd((uint64_t)hd.nnz * 4) == TCRNET_OK) h->d_cols = static_cast<int32_t*>(p);
    if (rd(n * 4) == TCRNET_OK) h->d_degree = static_cast<int32_t*>(p);
    if (hd.has_bucketed) {
        if (rd(n * sizeof(Canon)) == TCRNET_OK) h->d_bcanon = static_cast<Canon*>(p);
        if (rd(n * 4) == TCRNET_OK) h->d_bperm = static_cast<int32_t*>(p);
    }
    if (hd.has_input_order) {
        if (rd(n * sizeof(Canon)) == TCRNET_OK) h->d_canon_in = static_cast<Canon*>(p);
        if (rd(n) == TCRNET_OK) h->d_lens = static_cast<uint8_t*>(p);
    }
    if (hd.has_index) {
        // the index arrays are sized for n strings (ids >= U unused)
        DevBuf uc;
        if (st == TCRNET_OK) st = uc.alloc_owned(sizeof(Canon) * (n > 0 ? n : 1), s);
        if (st == TCRNET_OK) {
            uint64_t bytes = 0;
            const uint64_t want = (uint64_t)hd.ix_U * sizeof(Canon);
            if (std::fread(&bytes, sizeof(bytes), 1, f) != 1 || bytes != want) st = TCRNET_EINVAL;
            if (st == TCRNET_OK && bytes > 0) {
                buf.resize(bytes);
                if (std::fread(buf.data(), 1, bytes, f) != bytes) st = TCRNET_EINVAL;
                else if (cudaMemcpyAsync(uc.as<void>(), buf.data(), bytes, cudaMemcpyHostToDevice, s) != cudaSuccess ||
                         cudaStreamSynchronize(s) != cudaSuccess)
                    st = TCRNET_EDEVICE;
            }
            if (st == TCRNET_OK) h->ix.ucanon = static_cast<Canon*>(uc.release());
        }
        if (rd(n * 4) == TCRNET_OK) h->ix.umult = static_cast<int32_t*>(p);
        if (rd((n + 1) * 8) == TCRNET_OK) h->ix.mem_off = static_cast<int64_t*>(p);
        if (rd(n * 4) == TCRNET_OK) h->ix.members = static_cast<int32_t*>(p);
        if (rd((uint64_t)hd.ix_R * 8) == TCRNET_OK) h->ix.recs = static_cast<uint64_t*>(p);
        if (rd(((uint64_t)hd.ix_P + 1) * 8) == TCRNET_OK) h->ix.poff = static_cast<int64_t*>(p);
        if (hd.ix_E >= 0) {
            if (rd(n * 4) == TCRNET_OK) h->ix.uid = static_cast<int32_t*>(p);
            if (rd((uint64_t)hd.ix_E * 8) == TCRNET_OK) h->ix.uedges = static_cast<int2*>(p);
            h->ix.E = hd.ix_E;
        }
        h->ix.U = hd.ix_U;
        h->ix.P = hd.ix_P;
        h->ix.R = hd.ix_R;
        h->ix.n = hd.n;
    }
    std::fclose(f);
    if (st != TCRNET_OK) {
        cudaStreamSynchronize(s);
        free_handle_memory(h);
        delete h;
        return st;
    }
    *out = h;
    return TCRNET_OK;
}

tcrnet_status tcrnet_stats_get(tcrnet_handle h, tcrnet_stats* out) {
    if (!h || !out) return TCRNET_EINVAL;
    *out = h->stats;
    return TCRNET_OK;
}

void tcrnet_free(tcrnet_handle h) {
    if (!h) return;
    DeviceGuard dg;
    dg.set(h->device);
    free_handle_memory(h);  // every call on h already completed; see free_stream
    delete h;
}

const char* tcrnet_strerror(tcrnet_status s) {
    switch (s) {
        case TCRNET_OK: return "ok";
        case TCRNET_EINVAL: return "invalid argument (empty string, bad offsets or parameter)";
        case TCRNET_EBADCHAR: return "character outside the 20 standard amino acids";
        case TCRNET_ETOOLONG: return "string longer than TCRNET_MAX_LEN";
        case TCRNET_ENOTSUP: return "not supported (deletion method with threshold >= 2, or option)";
        case TCRNET_ENOMEM: return "out of memory";
        case TCRNET_EDEVICE: return "CUDA device error";
        case TCRNET_ETIMEOUT: return "bounded device wait timed out";
        case TCRNET_ESTATE: return "handle cannot serve this call";
        case TCRNET_ECAPACITY: return "input larger than this fixed-capacity entry point accepts";
        default: return "unknown status";
    }
}

int64_t tcrnet_last_error_index(void) { return t_last_bad; }

const char* tcrnet_version(void) { return "tcrnet 0.1 (sm_103a)"; }

const char* tcrnet_last_cuda_error(void) { return t_last_cuda; }

}  // extern "C"
