// Single-pass exclusive scan building blocks (decoupled look-back), shared by
// the generic scan (scan.cu) and the deletion build's fused size scans.
//
// A scan runs one block per tile of kScanTile items, tiles taken by ticket (an
// atomic counter) so that they start in order. Each block scans its tile,
// publishes the tile total, and one warp looks back over the preceding tiles'
// published words 32 at a time, adding tile totals until it meets a tile that
// has published its inclusive prefix; the block then publishes its own. A
// tile only waits on tiles with smaller tickets, which are already running and
// wait only on tiles before them, so every wait ends; each wait is still
// bounded (kMaxLookbackSpins), after which the warp sets an error flag and
// goes on.
#pragma once

#include "common.cuh"

namespace tcr {

// 256 threads x 16 items: a tile of 4096 items with few enough registers per
// block that every tile of a scan (and of two scans in one launch) is resident
// at once at N = 8e5, so no look-back waits on a tile of a later wave.
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;
// Tiles are staged in shared memory: loaded item by item across the threads
// (coalesced), read back as each thread's kScanItems consecutive items. One
// padding word after every 16 items keeps those reads to two-way bank
// conflicts (unpadded, every lane of a warp hit the same bank).
constexpr int kScanStage = kScanTile + kScanTile / 16;
__host__ __device__ constexpr int scan_slot(int i) { return i + (i >> 4); }

// Published word of a tile: flag in bits 63..62 (0 nothing yet, 1 tile total,
// 2 inclusive prefix through this tile), value in bits 61..0.
constexpr unsigned long long kFlagTotal = 1ull << 62;
constexpr unsigned long long kFlagIncl = 2ull << 62;
constexpr unsigned long long kValueMask = (1ull << 62) - 1;
constexpr int kMaxLookbackSpins = 1 << 22;

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Block-wide exclusive scan (kScanThreads threads) of one value per thread;
// returns the block total. warp_tot: 32 shared words.
__device__ __forceinline__ int64_t scan_block_exclusive(int64_t v, int64_t& excl, int64_t* warp_tot) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int64_t y = __shfl_up_sync(kFull, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t t = lane < (kScanThreads / 32) ? warp_tot[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int64_t y = __shfl_up_sync(kFull, t, d);
            if (lane >= d) t += y;
        }
        if (lane < (kScanThreads / 32)) warp_tot[lane] = t;  // inclusive warp totals
    }
    __syncthreads();
    const int64_t base = warp > 0 ? warp_tot[warp - 1] : 0;
    excl = base + x - v;
    const int64_t total = warp_tot[kScanThreads / 32 - 1];
    __syncthreads();
    return total;
}

// Publish tile `tile`'s total and find the sum of all earlier tiles; called by
// the block's first warp (all 32 lanes), which returns that sum in every lane.
// status[0 .. tiles) are the tiles' words, status[tiles + 1] the error flag.
__device__ __forceinline__ int64_t scan_lookback(int64_t tile, int64_t tot, unsigned long long* status,
                                                 int64_t tiles) {
    const int lane = threadIdx.x & 31;
    if (tile == 0) {
        if (lane == 0) st_release_u64(status, kFlagIncl | ((unsigned long long)tot & kValueMask));
        return 0;
    }
    if (lane == 0) st_release_u64(status + tile, kFlagTotal | ((unsigned long long)tot & kValueMask));
    int64_t prefix = 0;
    int64_t window = tile - 1;
    bool gave_up = false;
    while (true) {
        const int64_t j = window - lane;  // lane k reads tile (window - k)
        unsigned long long w = kFlagIncl;  // beyond tile 0: nothing to add
        if (j >= 0) {
            int spins = 0;
            while (((w = ld_acquire_u64(status + j)) >> 62) == 0) {
                if (++spins >= kMaxLookbackSpins) {
                    gave_up = true;
                    w = kFlagIncl;  // bounded: end the walk (the error flag is set below)
                    break;
                }
                __nanosleep(32);
            }
        }
        __syncwarp();
        // the nearest tile with an inclusive prefix ends the walk; the tiles
        // between it and this one add their totals
        const unsigned incl = __ballot_sync(kFull, (w >> 62) == 2);
        const int stop = incl ? __ffs(incl) - 1 : 32;
        int64_t add = (lane <= stop && j >= 0) ? (int64_t)(w & kValueMask) : 0;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) add += __shfl_xor_sync(kFull, add, d);
        prefix += add;
        if (incl) break;
        window -= 32;
    }
    if (__any_sync(kFull, gave_up) && lane == 0) atomicExch(status + tiles + 1, 1ull);
    if (lane == 0) st_release_u64(status + tile, kFlagIncl | ((unsigned long long)(prefix + tot) & kValueMask));
    return prefix;
}

}  // namespace tcr
