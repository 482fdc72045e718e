// Exclusive prefix sums (row counts -> CSR offsets) and offset helpers.
//
// One pass with decoupled look-back (lookback.cuh): one launch per scan, the
// input read once. Single-tile inputs take one block without look-back.
#include "kernels.cuh"
#include "lookback.cuh"

namespace tcr {
namespace {

template <typename TI>
__device__ __forceinline__ int64_t load_item(const TI* in, int64_t i, int64_t n) {
    return i < n ? (int64_t)in[i] : 0;
}

template <typename TI>
__global__ void __launch_bounds__(kScanThreads) k_tile_scan(const TI* __restrict__ in, int64_t n,
                                                             const int64_t* __restrict__ tile_base,
                                                             int64_t* __restrict__ out) {
    __shared__ int64_t warp_tot[32];
    __shared__ int64_t stage[kScanStage];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int idx = k * kScanThreads + threadIdx.x;
        stage[scan_slot(idx)] = load_item(in, base + idx, n);
    }
    __syncthreads();
    int64_t v[kScanItems];
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = stage[scan_slot(threadIdx.x * kScanItems + k)];
        s += v[k];
    }
    int64_t excl;
    int64_t tot = scan_block_exclusive(s, excl, warp_tot);
    int64_t run = excl + (tile_base ? tile_base[blockIdx.x] : 0);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        stage[scan_slot(threadIdx.x * kScanItems + k)] = run;
        run += v[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k * kScanThreads + threadIdx.x;
        if (i < n) out[i] = stage[scan_slot(k * kScanThreads + threadIdx.x)];
    }
    // the last tile also writes the grand total at out[n]
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = (tile_base ? tile_base[blockIdx.x] : 0) + tot;
}

// status[0 .. tiles) publication words, status[tiles] the ticket counter,
// status[tiles + 1] the error flag; all zero at launch.
// `clear` (nullable) may be `in` itself: neither is declared restrict, and
// each item is read into shared memory before it is overwritten: with zero,
// or with its exclusive prefix when `seed` is set.
template <typename TI>
__global__ void __launch_bounds__(kScanThreads) k_scan_onepass(const TI* in, int64_t n, int64_t* __restrict__ out,
                                                                unsigned long long* status, int64_t tiles,
                                                                TI* clear, bool seed = false) {
    dep_entry();  // launched dependent on the kernel before it
    __shared__ int64_t warp_tot[32];
    __shared__ int64_t stage[kScanStage];
    __shared__ int64_t s_prefix;
    __shared__ int64_t s_tile;
    if (threadIdx.x == 0) s_tile = (int64_t)atomicAdd(status + tiles, 1ull);
    __syncthreads();
    const int64_t tile = s_tile;
    const int64_t base = tile * kScanTile;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int idx = k * kScanThreads + threadIdx.x;
        stage[scan_slot(idx)] = load_item(in, base + idx, n);
    }
    if (clear && !seed) {  // in place of a memset before the input's next use as counters
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            const int64_t i = base + k * kScanThreads + threadIdx.x;
            if (i < n) clear[i] = 0;
        }
    }
    __syncthreads();
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
            if (seed) clear[i] = (TI)o;
        }
    }
    if (tile == tiles - 1 && threadIdx.x == 0) out[n] = s_prefix + tot;  // the grand total
}

__global__ void k_narrow(const int64_t* __restrict__ in, int32_t* __restrict__ out, int64_t count);

template <typename TI>
tcrnet_status scan_impl(const TI* in, int64_t* out, int64_t n, cudaStream_t s,
                        unsigned long long* zeroed_status = nullptr, bool clear_input = false, bool seed = false) {
    if (n <= 0) {
        TCR_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
        return TCRNET_OK;
    }
    const int64_t tiles = ceil_div(n, kScanTile);
    if (tiles == 1) {
        k_tile_scan<TI><<<1, kScanThreads, 0, s>>>(in, n, nullptr, out);
        TCR_LAUNCH_CHECK();
        if (seed) {
            if constexpr (sizeof(TI) == sizeof(int32_t)) {
                k_narrow<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(out, reinterpret_cast<int32_t*>(const_cast<TI*>(in)), n);
                TCR_LAUNCH_CHECK();
            } else {
                return TCRNET_EINVAL;
            }
        } else if (clear_input) {
            TCR_CUDA(cudaMemsetAsync(const_cast<TI*>(in), 0, sizeof(TI) * n, s));
        }
        return TCRNET_OK;
    }
    if (tiles > 0x7fffffffLL) return TCRNET_EINVAL;
    DevBuf status;
    unsigned long long* st = zeroed_status;
    if (!st) {
        TCR_CHECK(status.alloc(sizeof(unsigned long long) * (tiles + 2), s));
        TCR_CUDA(cudaMemsetAsync(status.as<void>(), 0, sizeof(unsigned long long) * (tiles + 2), s));
        st = status.as<unsigned long long>();
    }
    TCR_CUDA(launch_dependent(k_scan_onepass<TI>, dim3((unsigned)tiles), dim3(kScanThreads), 0, s, in, n, out, st,
                              tiles, (clear_input || seed) ? const_cast<TI*>(in) : nullptr, seed));
    note_launch();
    return TCRNET_OK;
}

__global__ void k_narrow(const int64_t* __restrict__ in, int32_t* __restrict__ out, int64_t count) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (int32_t)in[i];
}

__global__ void k_degree(const int64_t* __restrict__ off, int32_t* __restrict__ deg, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        deg[i] = (int32_t)(off[i + 1] - off[i]);
}

inline unsigned grid_for(int64_t n, int threads) {
    int64_t b = ceil_div(n, threads);
    if (b < 1) b = 1;
    if (b > 65535LL * 32) b = 65535LL * 32;
    return (unsigned)b;
}

}  // namespace

int64_t scan_status_words(int64_t n) {
    const int64_t tiles = ceil_div(n, kScanTile);
    return tiles > 1 ? tiles + 2 : 0;
}

tcrnet_status scan_exclusive_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s,
                                        unsigned long long* zeroed_status, bool clear_input) {
    return scan_impl<int32_t>(in, out, n, s, zeroed_status, clear_input);
}

tcrnet_status scan_exclusive_i32_to_i64_cursors(int32_t* in, int64_t* out, int64_t n, cudaStream_t s,
                                                unsigned long long* zeroed_status) {
    return scan_impl<int32_t>(in, out, n, s, zeroed_status, false, true);
}

tcrnet_status scan_exclusive_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s) {
    return scan_impl<int64_t>(in, out, n, s);
}

tcrnet_status narrow_offsets(const int64_t* in, int32_t* out, int64_t count, cudaStream_t s) {
    if (count <= 0) return TCRNET_OK;
    k_narrow<<<grid_for(count, 256), 256, 0, s>>>(in, out, count);
    TCR_LAUNCH_CHECK();
    return TCRNET_OK;
}

tcrnet_status degree_from_offsets(const int64_t* off, int32_t* degree, int64_t n, cudaStream_t s) {
    if (n <= 0) return TCRNET_OK;
    k_degree<<<grid_for(n, 256), 256, 0, s>>>(off, degree, n);
    TCR_LAUNCH_CHECK();
    return TCRNET_OK;
}

}  // namespace tcr
