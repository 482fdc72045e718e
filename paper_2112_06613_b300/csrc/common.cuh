// Shared definitions of the tcrnet CUDA library (sm_103a).
//
// Canonical string layout ("canon"): 5-bit amino-acid codes, 12 codes per
// 64-bit word, code k at word k / 12, bits 5 * (k % 12); four words hold the
// longest accepted string (48). Code 0 is padding, codes 1..20 are the 20
// standard amino acids in the order the paper lists the set Sigma (Methods
// "Combination of amino acids"): A R N D C Q E G H I L K M F P S T W Y V.
// The paper stores one byte per amino acid (Methods "GPU-based network
// generation"); 5-bit fields let one XOR compare six positions per 32-bit word.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <utility>
#include <vector>

#include "tcrnet.h"

namespace tcr {

constexpr int kMaxLen = TCRNET_MAX_LEN;  // 48
constexpr int kCodesPerWord = 12;
constexpr int kCanonWords = 4;
constexpr unsigned kFull = 0xffffffffu;

struct __align__(16) Canon {
    uint64_t w[kCanonWords];
};

// Bits 60..63 of the four words hold no code. A batched build stores the
// repertoire number there (16 bits, nibble k in word k), so strings of
// different repertoires never compare equal and never hash alike on purpose.
constexpr uint64_t kTagBits = 0xF000000000000000ULL;

// ASCII -> code (0 = not in the alphabet).
__host__ __device__ inline uint32_t aa_code(uint32_t c) {
    switch (c) {
        case 'A': return 1;  case 'R': return 2;  case 'N': return 3;  case 'D': return 4;
        case 'C': return 5;  case 'Q': return 6;  case 'E': return 7;  case 'G': return 8;
        case 'H': return 9;  case 'I': return 10; case 'L': return 11; case 'K': return 12;
        case 'M': return 13; case 'F': return 14; case 'P': return 15; case 'S': return 16;
        case 'T': return 17; case 'W': return 18; case 'Y': return 19; case 'V': return 20;
        default: return 0;
    }
}

__device__ __forceinline__ uint32_t canon_code(const Canon& c, int k) {
    return (uint32_t)(c.w[k / kCodesPerWord] >> (5 * (k % kCodesPerWord))) & 31u;
}

__device__ __forceinline__ Canon load_canon(const Canon* p) {
    const ulonglong2* q = reinterpret_cast<const ulonglong2*>(p);
    ulonglong2 x = __ldg(q);
    ulonglong2 y = __ldg(q + 1);
    Canon c;
    c.w[0] = x.x; c.w[1] = x.y; c.w[2] = y.x; c.w[3] = y.y;
    return c;
}

// Plain (coherent, any state space) load, e.g. from shared memory; load_canon
// above is for read-only global data only.
__device__ __forceinline__ Canon load_canon_plain(const Canon* p) {
    const ulonglong2* q = reinterpret_cast<const ulonglong2*>(p);
    const ulonglong2 x = q[0];
    const ulonglong2 y = q[1];
    Canon c;
    c.w[0] = x.x; c.w[1] = x.y; c.w[2] = y.x; c.w[3] = y.y;
    return c;
}

__device__ __forceinline__ void store_canon(Canon* p, const Canon& c) {
    ulonglong2* q = reinterpret_cast<ulonglong2*>(p);
    q[0] = make_ulonglong2(c.w[0], c.w[1]);
    q[1] = make_ulonglong2(c.w[2], c.w[3]);
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Append this lane's `k` hits (pairs (a, row_b[0..k)) given by emit) to a pair
// sink with one atomic per warp: every lane of the warp must call it (k may
// be 0). emit(slot_base) writes the lane's pairs at slots slot_base ..
// slot_base + k - 1 when they are below cap.
template <typename Emit>
__device__ __forceinline__ void warp_append_pairs(unsigned long long* cursor, int k, Emit emit) {
    const unsigned any = __ballot_sync(0xffffffffu, k > 0);
    if (!any) return;
    const int lane = threadIdx.x & 31;
    int x = k;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    const int total = __shfl_sync(0xffffffffu, x, 31);
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(cursor, (unsigned long long)total);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (k > 0) emit((long long)(base + (unsigned long long)(x - k)));
}

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Programmatic dependent launch (sm_90 and later). A kernel launched with
// launch_dependent() may be scheduled while the kernel before it on the
// stream is still finishing, which hides most of the launch gap between the
// two. Such a kernel calls dep_entry() before anything else: it waits until
// the kernel before it has completed and its writes are visible, then lets
// the kernel after it be scheduled in turn. Launched normally, dep_entry()
// returns at once, so a kernel may be launched either way.
__device__ __forceinline__ void dep_entry() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_dependent(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                    Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Error record of the last failing CUDA call (diagnostics only).
void note_cuda_error(cudaError_t e, const char* what, const char* file, int line);

inline tcrnet_status status_of(cudaError_t e) {
    if (e == cudaSuccess) return TCRNET_OK;
    if (e == cudaErrorMemoryAllocation) return TCRNET_ENOMEM;
    return TCRNET_EDEVICE;
}

#define TCR_CUDA(call)                                                  \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) {                                        \
            ::tcr::note_cuda_error(e_, #call, __FILE__, __LINE__);      \
            if (e_ == cudaErrorMemoryAllocation) (void)cudaGetLastError(); \
            return ::tcr::status_of(e_);                                \
        }                                                               \
    } while (0)

#define TCR_CHECK(expr)                                                 \
    do {                                                                \
        tcrnet_status s_ = (expr);                                      \
        if (s_ != TCRNET_OK) return s_;                                 \
    } while (0)

// Counts kernel launches of the calling thread (reported in tcrnet_stats).
void note_launch();
int64_t launches_so_far();

#define TCR_LAUNCH_CHECK()      \
    do {                        \
        ::tcr::note_launch();   \
        TCR_CUDA(cudaGetLastError()); \
    } while (0)

// Build workspace: scratch memory of a build or query is carved from a
// per-device arena of cached chunks (a bump allocator reset at the start of
// every call), so a call in steady state makes no allocator calls for its
// scratch. A call leases the arena for its duration (ArenaLease); if another
// host thread holds it, the call falls back to stream-ordered allocations.
// Buffers handed to a handle are never carved from the arena.
void* arena_carve(size_t bytes, cudaError_t* err);  // nullptr: no lease on this thread
bool arena_active();
// While the calling thread holds its device's workspace lease: a second stream
// of that device and events for forking independent work off the call's
// stream and joining it back (null: no lease; run everything in order).
// ev[0..3] and ev[6] belong to the deletion build's phases, ev[4], ev[5] and
// ev[7] to the row sort; stream2 is a third stream the row sort uses when its
// long classes are listed in advance.
struct SideStream {
    cudaStream_t stream = nullptr;
    cudaStream_t stream2 = nullptr;
    cudaEvent_t ev[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
};
const SideStream* leased_side_stream();

// Page-locked host memory of the calling thread (kPinnedScratchBytes,
// allocated on first use and kept for the thread's life) for small
// device-to-host readbacks of counters, sizes and error words. Copies into it
// are asynchronous, so a group of readbacks costs one stream synchronisation;
// a copy into pageable memory waits for the device on its own (measured: four
// pageable readbacks in a row left the GPU idle for ~80 us mid-build).
// nullptr if page-locked memory cannot be had (callers fall back to pageable).
constexpr size_t kPinnedScratchBytes = 4096;
void* pinned_scratch();
// The same memory as a device address (it is mapped), so a kernel can write a
// group of readback values there directly: one small kernel instead of one
// copy per value. nullptr if unavailable.
void* pinned_scratch_device();
// count small device values (bytes[k] bytes from device address src[k] to host
// address dst[k]) read back with one stream synchronisation, through the
// page-locked scratch (pageable copies when it cannot be had or the values do
// not fit in it).
tcrnet_status read_back(cudaStream_t s, int count, const void* const* src, void* const* dst, const size_t* bytes);

// Events for the optional phase timing, recycled through a per-device pool so
// that a profiled build does not create and destroy events on its critical path.
cudaEvent_t event_acquire();          // an event of the current device
void event_release(cudaEvent_t e);    // back to the current device's pool

// CUDA-event marks on one stream (no-op when off); ms(a, b) waits for mark b.
class EventMarks {
public:
    EventMarks(bool on, cudaStream_t s) : on_(on), s_(s) {}
    ~EventMarks() {
        for (auto e : ev_) event_release(e);
    }
    EventMarks(const EventMarks&) = delete;
    EventMarks& operator=(const EventMarks&) = delete;
    int mark() {
        if (!on_) return -1;
        cudaEvent_t e = event_acquire();
        if (!e) return -1;
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

class ArenaLease {
public:
    ArenaLease(int device, cudaStream_t s);
    ~ArenaLease();
    ArenaLease(const ArenaLease&) = delete;
    ArenaLease& operator=(const ArenaLease&) = delete;

private:
    int dev_ = -1;
    cudaStream_t s_ = 0;
    bool held_ = false;
};

// Device buffer: arena scratch while a lease is active on this thread
// (alloc), otherwise stream-ordered cudaMallocAsync / cudaFreeAsync; alloc_owned
// always allocates (for results a handle keeps). Freed when it goes out of
// scope unless released.
// Host-side fault injection (options.fail_alloc_at): when armed, the k-th
// allocation of the calling thread's current call fails with ENOMEM.
bool alloc_fault_tick();  // true: fail this allocation

class AllocFaultScope {
public:
    explicit AllocFaultScope(int32_t fail_at);
    ~AllocFaultScope();
    AllocFaultScope(const AllocFaultScope&) = delete;
    AllocFaultScope& operator=(const AllocFaultScope&) = delete;

private:
    int64_t saved_;
};

class DevBuf {
public:
    // Large blocks are requested in size classes (multiples of an eighth of
    // their power of two, at most 12.5% over): a network that grows by small
    // inserts then gets a block of the size that its previous version freed,
    // which the stream-ordered pool reuses, instead of a slightly larger one
    // that would map new memory on every insert.
    static size_t size_class(size_t bytes) {
        if (bytes < (size_t(32) << 20)) return bytes;
        int top = 63 - __builtin_clzll((unsigned long long)bytes);
        const size_t step = size_t(1) << (top - 3);
        return (bytes + step - 1) / step * step;
    }
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    DevBuf(DevBuf&& o) noexcept : p_(o.p_), bytes_(o.bytes_), s_(o.s_), arena_(o.arena_) {
        o.p_ = nullptr;
        o.bytes_ = 0;
    }
    DevBuf& operator=(DevBuf&& o) noexcept {
        if (this != &o) {
            reset();
            p_ = o.p_;
            bytes_ = o.bytes_;
            s_ = o.s_;
            arena_ = o.arena_;
            o.p_ = nullptr;
            o.bytes_ = 0;
        }
        return *this;
    }
    ~DevBuf() { reset(); }
    tcrnet_status alloc(size_t bytes, cudaStream_t s) {
        if (alloc_fault_tick()) {
            reset();
            return TCRNET_ENOMEM;
        }
        if (arena_active()) {
            reset();
            cudaError_t e = cudaSuccess;
            void* p = arena_carve(bytes == 0 ? 16 : bytes, &e);
            if (!p) {
                note_cuda_error(e, "arena chunk", __FILE__, __LINE__);
                (void)cudaGetLastError();
                return status_of(e == cudaSuccess ? cudaErrorMemoryAllocation : e);
            }
            p_ = p;
            bytes_ = bytes;
            s_ = s;
            arena_ = true;
            return TCRNET_OK;
        }
        return owned_alloc(bytes, s);
    }
    tcrnet_status alloc_owned(size_t bytes, cudaStream_t s) {
        reset();
        if (alloc_fault_tick()) return TCRNET_ENOMEM;
        return owned_alloc(bytes, s);
    }
    tcrnet_status owned_alloc(size_t bytes, cudaStream_t s) {
        reset();
        s_ = s;
        bytes_ = bytes;
        arena_ = false;
        if (bytes == 0) bytes = 16;
        cudaError_t e = cudaMallocAsync(&p_, size_class(bytes), s);
        if (e != cudaSuccess) {
            p_ = nullptr;
            bytes_ = 0;
            note_cuda_error(e, "cudaMallocAsync", __FILE__, __LINE__);
            (void)cudaGetLastError();
            return status_of(e);
        }
        return TCRNET_OK;
    }
    void reset() {
        if (p_ && !arena_) cudaFreeAsync(p_, s_);
        p_ = nullptr;
        bytes_ = 0;
        arena_ = false;
    }
    // Hand the allocation to its new owner; arena scratch cannot be handed out.
    void* release() {
        if (arena_) return nullptr;
        void* p = p_;
        p_ = nullptr;
        bytes_ = 0;
        return p;
    }
    template <typename T>
    T* as() const { return static_cast<T*>(p_); }
    size_t bytes() const { return bytes_; }

private:
    void* p_ = nullptr;
    size_t bytes_ = 0;
    cudaStream_t s_ = 0;
    bool arena_ = false;
};

}  // namespace tcr
