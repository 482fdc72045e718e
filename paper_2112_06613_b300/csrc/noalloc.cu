// Node degrees without any device allocation (tcrnet_degree_noalloc).
//
// Some callers cannot call cudaMalloc: applications whose device memory was
// handed in full to another allocator at start-up (a caching pool that
// reserves all free memory), and services that forbid device allocation after
// start-up because an allocation can synchronise the device or map pages and
// so break their latency bound. This entry point serves them for small
// repertoires: it is a variant of the pair test count pass that needs no
// workspace from the caller or from the allocator. Its working memory (the
// packed strings, their lengths and an error word) lives in one fixed-size
// file-scope device array, g_noalloc_scratch, which every device that loads
// the library keeps until the process exits (about 0.5 MB).
//
// The caller passes device inputs (chars, offsets) and a device output
// (degree). Each call first clears the error word and the output, then packs
// the strings into the array, then counts, for every node, the other nodes
// within Levenshtein distance <= threshold with the same closed forms as the
// tile kernel: equal lengths -> at most `threshold` mismatching positions;
// lengths L, L+1 (threshold 1) -> the first mismatch of the shorter string
// against the longer lies after the last mismatch against the longer string
// shifted down by one position (longest common prefix + longest common suffix
// >= L), found with count-leading/trailing-zero instructions on the packed
// 64-bit words.
//
// All calls share the one array and it keeps the last call's contents, so
// calls that overlap on the GPU (different streams, different host threads)
// race and must be serialised by the caller. The array's device address is
// looked up once per device and kept for the process: after cudaDeviceReset
// of a device this entry point must not be called on it again.
#include <mutex>

#include "common.cuh"

namespace tcr {
namespace {

constexpr int64_t kNoAllocMaxN = TCRNET_NOALLOC_MAX_N;
constexpr size_t kCanonBytes = sizeof(Canon) * kNoAllocMaxN;
constexpr size_t kLenBytes = kNoAllocMaxN;
constexpr size_t kErrOffset = kCanonBytes + kLenBytes;  // multiple of 8
constexpr size_t kScratchBytes = kErrOffset + sizeof(unsigned long long);

// Working memory of tcrnet_degree_noalloc (see the file comment).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kThreads = 256;
constexpr int kColChunk = 2048;  // columns per block row (grid y)

// bit 4 and bit 0 of each of the twelve 5-bit fields of a canonical word
constexpr uint64_t kHI64 = 0x0842108421084210ULL;
constexpr uint64_t kLOW64 = 0x0084210842108421ULL;

struct View {
    Canon* canon;
    uint8_t* len;
    unsigned long long* err;
};

__host__ __device__ inline View view_of(unsigned char* base) {
    View v;
    v.canon = reinterpret_cast<Canon*>(base);
    v.len = base + kCanonBytes;
    v.err = reinterpret_cast<unsigned long long*>(base + kErrOffset);
    return v;
}

__device__ __forceinline__ uint64_t field_mismatch64(uint64_t x) {
    return (((x | kHI64) - kLOW64) | x) & kHI64;
}

__global__ void k_na_reset(unsigned char* scratch, int32_t* __restrict__ degree, int64_t n) {
    const View v = view_of(scratch);
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *v.err = ~0ull;
    if (i < n) degree[i] = 0;
}

__global__ void k_na_encode(const uint8_t* __restrict__ chars, const int64_t* __restrict__ offs, int64_t n,
                            unsigned char* scratch) {
    const View v = view_of(scratch);
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t s = offs[i];
    const int64_t len = offs[i + 1] - s;
    unsigned code_err = 0;
    Canon c;
    c.w[0] = c.w[1] = c.w[2] = c.w[3] = 0;
    if (len <= 0) {
        code_err = TCRNET_EINVAL;
    } else if (len > kMaxLen) {
        code_err = TCRNET_ETOOLONG;
    } else {
#pragma unroll
        for (int k = 0; k < kMaxLen; ++k) {
            if (k < len) {
                const uint64_t code = aa_code(chars[s + k]);
                if (code == 0) code_err = TCRNET_EBADCHAR;
                c.w[k / kCodesPerWord] |= code << (5 * (k % kCodesPerWord));
            }
        }
    }
    if (code_err) {
        atomicMin(v.err, ((unsigned long long)i << 8) | code_err);
        v.len[i] = 0;
    } else {
        store_canon(v.canon + i, c);
        v.len[i] = (uint8_t)len;
    }
}

__device__ __forceinline__ bool within(const Canon& a, int la, const Canon& b, int lb, int T) {
    if (la == lb) {
        int mism = 0;
#pragma unroll
        for (int w = 0; w < kCanonWords; ++w) mism += __popcll(field_mismatch64(a.w[w] ^ b.w[w]));
        return mism <= T;
    }
    if (T < 1) return false;
    // a shorter (length la), b longer (la + 1)
    const Canon& s = la < lb ? a : b;
    const Canon& l = la < lb ? b : a;
    int first = 4 * kCodesPerWord;  // first mismatch of s vs l
#pragma unroll
    for (int w = kCanonWords - 1; w >= 0; --w) {
        const uint64_t m = field_mismatch64(s.w[w] ^ l.w[w]);
        if (m) first = w * kCodesPerWord + (__ffsll((long long)m) - 1 - 4) / 5;
    }
    int last = -1;  // last mismatch of s vs l shifted down by one position
#pragma unroll
    for (int w = 0; w < kCanonWords; ++w) {
        const uint64_t next = (w + 1 < kCanonWords) ? (l.w[w + 1] & 31ull) : 0ull;
        const uint64_t down = (l.w[w] >> 5) | (next << 55);
        const uint64_t m = field_mismatch64(s.w[w] ^ down);
        if (m) last = w * kCodesPerWord + (63 - __clzll((long long)m) - 4) / 5;
    }
    return first > last;
}

__global__ void __launch_bounds__(kThreads)
k_na_degree(unsigned char* scratch, int64_t n, int T, int32_t* __restrict__ degree) {
    const View v = view_of(scratch);
    if (*v.err != ~0ull) return;  // bad input: the host reports it
    __shared__ Canon sc[kThreads];
    __shared__ uint8_t sl[kThreads];
    const int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    const bool row_ok = i < n;
    Canon a;
    int la = 0;
    if (row_ok) {
        a = load_canon(v.canon + i);
        la = v.len[i];
    }
    const int64_t c0 = (int64_t)blockIdx.y * kColChunk;
    const int64_t c1 = (c0 + kColChunk < n) ? (c0 + kColChunk) : n;
    int32_t cnt = 0;
    for (int64_t j0 = c0; j0 < c1; j0 += kThreads) {
        __syncthreads();
        const int64_t j = j0 + threadIdx.x;
        if (j < c1) {
            sc[threadIdx.x] = load_canon(v.canon + j);
            sl[threadIdx.x] = v.len[j];
        }
        __syncthreads();
        const int nb = (c1 - j0 < kThreads) ? (int)(c1 - j0) : kThreads;
        if (row_ok) {
            for (int k = 0; k < nb; ++k) {
                const int lb = sl[k];
                const int d = la - lb;
                if (d > T || -d > T || j0 + k == i) continue;
                cnt += within(a, la, sc[k], lb, T) ? 1 : 0;
            }
        }
    }
    if (row_ok && cnt) atomicAdd(&degree[i], cnt);
}

// Device address of g_noalloc_scratch, looked up once per device.
tcrnet_status scratch_address(int dev, unsigned char** out) {
    static std::mutex mu;
    static unsigned char* addr[64] = {nullptr};
    if (dev < 0 || dev >= 64) return TCRNET_EDEVICE;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            note_cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)", __FILE__, __LINE__);
            return TCRNET_EDEVICE;
        }
        addr[dev] = static_cast<unsigned char*>(p);
    }
    *out = addr[dev];
    return TCRNET_OK;
}

}  // namespace
}  // namespace tcr

extern "C" tcrnet_status tcrnet_degree_noalloc(const uint8_t* d_chars, const int64_t* d_offsets, int64_t n,
                                               int32_t threshold, int32_t* d_degree, void* stream,
                                               int64_t* bad_index) {
    using namespace tcr;
    if (bad_index) *bad_index = -1;
    if (n < 0 || threshold < 0) return TCRNET_EINVAL;
    if (threshold > 1) return TCRNET_ENOTSUP;
    if (n > kNoAllocMaxN) return TCRNET_ECAPACITY;
    if (n == 0) return TCRNET_OK;
    if (!d_chars || !d_offsets || !d_degree) return TCRNET_EINVAL;
    int dev = 0;
    TCR_CUDA(cudaGetDevice(&dev));
    unsigned char* scratch = nullptr;
    TCR_CHECK(scratch_address(dev, &scratch));
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned blocks = (unsigned)ceil_div(n, kThreads);
    k_na_reset<<<blocks, kThreads, 0, s>>>(scratch, d_degree, n);
    TCR_CUDA(cudaGetLastError());
    k_na_encode<<<blocks, kThreads, 0, s>>>(d_chars, d_offsets, n, scratch);
    TCR_CUDA(cudaGetLastError());
    const dim3 grid(blocks, (unsigned)ceil_div(n, kColChunk));
    k_na_degree<<<grid, kThreads, 0, s>>>(scratch, n, threshold, d_degree);
    TCR_CUDA(cudaGetLastError());
    unsigned long long h_err = ~0ull;
    TCR_CUDA(cudaMemcpyAsync(&h_err, view_of(scratch).err, sizeof(h_err), cudaMemcpyDeviceToHost, s));
    TCR_CUDA(cudaStreamSynchronize(s));
    if (h_err != ~0ull) {
        if (bad_index) *bad_index = (int64_t)(h_err >> 8);
        return (tcrnet_status)(h_err & 0xff);
    }
    return TCRNET_OK;
}
