// Exclusive prefix sums (row counts -> CSR offsets) and offset helpers.
//
// Three phases: per-tile totals, a scan of the tile totals (recursive), and a
// rescan of each tile with its base added. Tiles are 4096 items, 512 threads,
// 8 contiguous items per thread staged through shared memory so global
// accesses stay coalesced.
#include "kernels.cuh"

namespace tcr {
namespace {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

template <typename TI>
__device__ __forceinline__ int64_t load_item(const TI* in, int64_t i, int64_t n) {
    return i < n ? (int64_t)in[i] : 0;
}

// Block-wide exclusive scan of one value per thread; returns the block total.
__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t& excl, int64_t* warp_tot) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int64_t y = __shfl_up_sync(kFull, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t t = lane < (kScanThreads / 32) ? warp_tot[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            int64_t y = __shfl_up_sync(kFull, t, d);
            if (lane >= d) t += y;
        }
        if (lane < (kScanThreads / 32)) warp_tot[lane] = t;  // inclusive warp totals
    }
    __syncthreads();
    int64_t base = warp > 0 ? warp_tot[warp - 1] : 0;
    excl = base + x - v;
    int64_t total = warp_tot[kScanThreads / 32 - 1];
    __syncthreads();
    return total;
}

template <typename TI>
__global__ void __launch_bounds__(kScanThreads) k_tile_totals(const TI* __restrict__ in, int64_t n,
                                                               int64_t* __restrict__ totals) {
    __shared__ int64_t warp_tot[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) s += load_item(in, base + k * kScanThreads + threadIdx.x, n);
    int64_t excl;
    int64_t tot = block_exclusive_scan(s, excl, warp_tot);
    if (threadIdx.x == 0) totals[blockIdx.x] = tot;
}

template <typename TI>
__global__ void __launch_bounds__(kScanThreads) k_tile_scan(const TI* __restrict__ in, int64_t n,
                                                             const int64_t* __restrict__ tile_base,
                                                             int64_t* __restrict__ out) {
    __shared__ int64_t warp_tot[32];
    __shared__ int64_t stage[kScanTile];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int idx = k * kScanThreads + threadIdx.x;
        stage[idx] = load_item(in, base + idx, n);
    }
    __syncthreads();
    int64_t v[kScanItems];
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = stage[threadIdx.x * kScanItems + k];
        s += v[k];
    }
    int64_t excl;
    int64_t tot = block_exclusive_scan(s, excl, warp_tot);
    int64_t run = excl + (tile_base ? tile_base[blockIdx.x] : 0);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        stage[threadIdx.x * kScanItems + k] = run;
        run += v[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k * kScanThreads + threadIdx.x;
        if (i < n) out[i] = stage[k * kScanThreads + threadIdx.x];
    }
    // the last tile also writes the grand total at out[n]
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = (tile_base ? tile_base[blockIdx.x] : 0) + tot;
}

template <typename TI>
tcrnet_status scan_impl(const TI* in, int64_t* out, int64_t n, cudaStream_t s) {
    if (n <= 0) {
        TCR_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
        return TCRNET_OK;
    }
    int64_t tiles = ceil_div(n, kScanTile);
    if (tiles == 1) {
        k_tile_scan<TI><<<1, kScanThreads, 0, s>>>(in, n, nullptr, out);
        TCR_LAUNCH_CHECK();
        return TCRNET_OK;
    }
    DevBuf totals, bases;
    TCR_CHECK(totals.alloc(sizeof(int64_t) * tiles, s));
    TCR_CHECK(bases.alloc(sizeof(int64_t) * (tiles + 1), s));
    k_tile_totals<TI><<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, totals.as<int64_t>());
    TCR_LAUNCH_CHECK();
    TCR_CHECK(scan_impl<int64_t>(totals.as<int64_t>(), bases.as<int64_t>(), tiles, s));
    k_tile_scan<TI><<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, bases.as<int64_t>(), out);
    TCR_LAUNCH_CHECK();
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

tcrnet_status scan_exclusive_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s) {
    return scan_impl<int32_t>(in, out, n, s);
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
