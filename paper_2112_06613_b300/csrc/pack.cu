// Validate, encode and length-bucket the input strings (the amino-acid alphabet
// Sigma of Methods "Combination of amino acids", one code per letter).
//
// The paper keeps each amino acid as one byte in a 30-slot buffer (Methods
// "GPU-based network generation"); here each string becomes the 32-byte
// canonical 5-bit form. Strings are then placed in buckets by length with a
// stable counting sort (input order is kept inside a bucket), because only
// strings whose lengths differ by at most l_max can be within distance l_max
// (lev >= |len a - len b|), so the pair kernels only visit bucket pairs
// (L, L) and (L, L + 1).
//
// k_encode: one thread per string. Reads its bytes, maps them through a
//   shared-memory table, packs the codes, and counts lengths per block into
//   blockcnt[len * nblocks + block] (length-major, so one exclusive scan over
//   the whole array yields every block's first slot in every bucket).
// k_bucket_scatter: recomputes each string's rank among equal-length strings
//   of its block (warp match_any + popc, then a per-warp prefix) and writes the
//   bucket-ordered copy plus the bucket position -> input index map.
#include "kernels.cuh"

namespace tcr {
namespace {

constexpr int kPackThreads = 256;
constexpr int kPackWarps = kPackThreads / 32;
constexpr int kBins = kMaxLen + 1;

__global__ void __launch_bounds__(kPackThreads)
k_encode(const uint8_t* __restrict__ chars, const int64_t* __restrict__ offs, int64_t n, int64_t lo, int64_t hi,
         Canon* __restrict__ canon, uint8_t* __restrict__ lens, int32_t* __restrict__ blockcnt,
         int nblocks, unsigned long long* __restrict__ err, unsigned long long* __restrict__ lensum) {
    __shared__ uint8_t lut[256];
    __shared__ int cnt[kBins];
    for (int t = threadIdx.x; t < 256; t += blockDim.x) lut[t] = (uint8_t)aa_code((uint32_t)t);
    for (int t = threadIdx.x; t < kBins; t += blockDim.x) cnt[t] = 0;
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * kPackThreads + threadIdx.x;
    int bin = -1;  // length of a valid string (counted below), -1 otherwise
    if (i < n) {
        const int64_t s = offs[i];
        const int64_t len = offs[i + 1] - s;
        unsigned code_err = 0;
        Canon c;
        c.w[0] = c.w[1] = c.w[2] = c.w[3] = 0;
        // empty, decreasing offsets, or outside the uploaded bytes (host inputs:
        // lo = first byte, hi = one past the last; device inputs: no bounds)
        const bool outside = lo != INT64_MIN && (s < lo || s > hi || len > hi - s);
        if (len <= 0 || outside) {
            code_err = TCRNET_EINVAL;
        } else if (len > kMaxLen) {
            code_err = TCRNET_ETOOLONG;
        } else {
            const uint8_t* p = chars + s;
            // word by word, up to the last word the string reaches (a 14-letter
            // string decodes 24 positions, not 48)
            const int ilen = (int)len;
#pragma unroll
            for (int w = 0; w < kCanonWords; ++w) {
                if (w * kCodesPerWord < ilen) {
                    uint64_t acc = 0;
#pragma unroll
                    for (int j = 0; j < kCodesPerWord; ++j) {
                        const int k = w * kCodesPerWord + j;
                        if (k < ilen) {
                            const uint64_t v = lut[p[k]];
                            if (v == 0) code_err = TCRNET_EBADCHAR;
                            acc |= v << (5 * j);
                        }
                    }
                    c.w[w] = acc;
                }
            }
        }
        if (code_err) {
            // the first error word holds the complement of (index << 8 | status)
            // so that zero means "none" and the lowest index wins by atomicMax
            atomicMax(err, ~(((unsigned long long)i << 8) | code_err));
            lens[i] = 0;
        } else {
            store_canon(canon + i, c);
            lens[i] = (uint8_t)len;
            bin = (int)len;
        }
    }
    // lengths cluster on a few values: one shared-memory add per length per warp
    const unsigned peers = __match_any_sync(kFull, bin);
    if (bin >= 0 && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&cnt[bin], __popc(peers));
    __syncthreads();
    if (blockcnt)
        for (int t = threadIdx.x; t < kBins; t += blockDim.x) blockcnt[(int64_t)t * nblocks + blockIdx.x] = cnt[t];
    if (threadIdx.x == 0) {
        unsigned long long total = 0;
        for (int t = 1; t < kBins; ++t) total += (unsigned long long)t * (unsigned long long)cnt[t];
        if (total) atomicAdd(lensum, total);
    }
}

__global__ void __launch_bounds__(kPackThreads)
k_bucket_scatter(const Canon* __restrict__ canon_in, const uint8_t* __restrict__ lens, int64_t n,
                 const int64_t* __restrict__ blockoff, int nblocks, Canon* __restrict__ canon_out,
                 int32_t* __restrict__ perm) {
    __shared__ int wcnt[kPackWarps][kBins];
    const int warp = threadIdx.x >> 5;
    for (int t = threadIdx.x; t < kPackWarps * kBins; t += blockDim.x) (&wcnt[0][0])[t] = 0;
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * kPackThreads + threadIdx.x;
    const int len = i < n ? (int)lens[i] : kBins;  // kBins = "no string"
    const unsigned peers = __match_any_sync(kFull, len);
    const int rank = __popc(peers & lanemask_lt());
    if (len < kBins && rank == 0) wcnt[warp][len] = __popc(peers);
    __syncthreads();
    if (len < kBins) {
        int pre = 0;
        for (int w = 0; w < warp; ++w) pre += wcnt[w][len];
        const int64_t pos = blockoff[(int64_t)len * nblocks + blockIdx.x] + pre + rank;
        store_canon(canon_out + pos, load_canon(canon_in + i));
        perm[pos] = (int32_t)i;
    }
}

// Repertoire tags of a batched build: string i of repertoire r gets r in the
// spare bits (nibble k of r in bits 60..63 of word k).
__global__ void k_tag(Canon* __restrict__ canon, int64_t n, const int64_t* __restrict__ rep_off, int64_t nrep) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t lo = 0, hi = nrep;  // largest r with rep_off[r] <= i
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (rep_off[mid] <= i) lo = mid; else hi = mid;
    }
    const uint64_t r = (uint64_t)lo;
    Canon c = load_canon_plain(canon + i);  // read and rewritten here: no read-only path
#pragma unroll
    for (int k = 0; k < kCanonWords; ++k) c.w[k] = (c.w[k] & ~kTagBits) | (((r >> (4 * k)) & 0xFull) << 60);
    store_canon(canon + i, c);
}

// Length counts per block of already encoded strings (lens).
__global__ void __launch_bounds__(kPackThreads)
k_count_lengths(const uint8_t* __restrict__ lens, int64_t n, int32_t* __restrict__ blockcnt, int nblocks) {
    __shared__ int cnt[kBins];
    for (int t = threadIdx.x; t < kBins; t += blockDim.x) cnt[t] = 0;
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * kPackThreads + threadIdx.x;
    if (i < n) atomicAdd(&cnt[lens[i]], 1);
    __syncthreads();
    for (int t = threadIdx.x; t < kBins; t += blockDim.x) blockcnt[(int64_t)t * nblocks + blockIdx.x] = cnt[t];
}

// Input order from bucket order: canon_in[perm[pos]] = canon[pos], lens from the bucket bounds.
__global__ void k_unbucket(const Canon* __restrict__ canon, const int32_t* __restrict__ perm, int64_t n,
                           const int64_t* __restrict__ bounds, Canon* __restrict__ canon_in, uint8_t* __restrict__ lens) {
    const int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= n) return;
    int L = 0;
    while (L < kMaxLen && bounds[L + 1] <= pos) ++L;
    const int32_t i = perm[pos];
    store_canon(canon_in + i, load_canon(canon + pos));
    lens[i] = (uint8_t)L;
}

__global__ void k_bucket_bounds(const int64_t* __restrict__ blockoff, int nblocks, int64_t* __restrict__ bounds) {
    const int t = threadIdx.x;
    if (t <= kBins) bounds[t] = blockoff[(int64_t)t * nblocks];  // t == kBins: the grand total
}

}  // namespace

tcrnet_status tag_repertoires(Canon* canon, int64_t n, const int64_t* rep_off_host, int64_t nrep, cudaStream_t s) {
    if (n == 0) return TCRNET_OK;
    DevBuf d;
    TCR_CHECK(d.alloc(sizeof(int64_t) * (nrep + 1), s));
    TCR_CUDA(cudaMemcpyAsync(d.as<void>(), rep_off_host, sizeof(int64_t) * (nrep + 1), cudaMemcpyHostToDevice, s));
    k_tag<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(canon, n, d.as<int64_t>(), nrep);
    TCR_LAUNCH_CHECK();
    TCR_CUDA(cudaStreamSynchronize(s));  // rep_off_host may go away
    return TCRNET_OK;
}

tcrnet_status bucket_from(const Canon* canon_in, const uint8_t* lens, int64_t n, Packed& out, cudaStream_t s) {
    for (int L = 0; L < kMaxLen + 2; ++L) out.bucket_off[L] = 0;
    if (n == 0) return TCRNET_OK;
    const int nblocks = (int)ceil_div(n, kPackThreads);
    TCR_CHECK(out.canon.alloc_owned(sizeof(Canon) * n, s));
    TCR_CHECK(out.perm.alloc_owned(sizeof(int32_t) * n, s));
    const int64_t ncnt = (int64_t)kBins * nblocks;
    DevBuf blockcnt, blockoff, bounds;
    TCR_CHECK(blockcnt.alloc(sizeof(int32_t) * ncnt, s));
    TCR_CHECK(blockoff.alloc(sizeof(int64_t) * (ncnt + 1), s));
    TCR_CHECK(bounds.alloc(sizeof(int64_t) * (kBins + 1), s));
    k_count_lengths<<<nblocks, kPackThreads, 0, s>>>(lens, n, blockcnt.as<int32_t>(), nblocks);
    TCR_LAUNCH_CHECK();
    TCR_CHECK(scan_exclusive_i32_to_i64(blockcnt.as<int32_t>(), blockoff.as<int64_t>(), ncnt, s));
    k_bucket_bounds<<<1, 64, 0, s>>>(blockoff.as<int64_t>(), nblocks, bounds.as<int64_t>());
    TCR_LAUNCH_CHECK();
    int64_t h_bounds[kBins + 1];
    TCR_CUDA(cudaMemcpyAsync(h_bounds, bounds.as<void>(), sizeof(h_bounds), cudaMemcpyDeviceToHost, s));
    k_bucket_scatter<<<nblocks, kPackThreads, 0, s>>>(canon_in, lens, n, blockoff.as<int64_t>(), nblocks,
                                                      out.canon.as<Canon>(), out.perm.as<int32_t>());
    TCR_LAUNCH_CHECK();
    TCR_CUDA(cudaStreamSynchronize(s));
    for (int L = 0; L <= kBins; ++L) out.bucket_off[L] = h_bounds[L];
    return TCRNET_OK;
}

tcrnet_status bucket_strings(Packed& out, cudaStream_t s) {
    return bucket_from(out.canon_in.as<Canon>(), out.lens.as<uint8_t>(), out.n, out, s);
}

tcrnet_status unbucket_strings(const Canon* canon, const int32_t* perm, const int64_t* bucket_off_host, int64_t n,
                               Canon* canon_in, uint8_t* lens, cudaStream_t s) {
    if (n == 0) return TCRNET_OK;
    DevBuf bounds;
    TCR_CHECK(bounds.alloc(sizeof(int64_t) * (kBins + 1), s));
    TCR_CUDA(cudaMemcpyAsync(bounds.as<void>(), bucket_off_host, sizeof(int64_t) * (kBins + 1), cudaMemcpyHostToDevice, s));
    k_unbucket<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(canon, perm, n, bounds.as<int64_t>(), canon_in, lens);
    TCR_LAUNCH_CHECK();
    return TCRNET_OK;
}

tcrnet_status pack_flags_status(unsigned long long first_error, int64_t* bad_index) {
    if (first_error == 0) return TCRNET_OK;
    const unsigned long long v = ~first_error;
    *bad_index = (int64_t)(v >> 8);
    return (tcrnet_status)(v & 0xff);
}

tcrnet_status pack_strings(const uint8_t* d_chars, const int64_t* d_offsets, int64_t n, Packed& out,
                           int64_t* bad_index, cudaStream_t s, bool bucket, bool keep_input_order, int64_t lo,
                           int64_t hi, bool defer_check) {
    out.n = n;
    out.lensum = 0;
    *bad_index = -1;
    for (int L = 0; L < kMaxLen + 2; ++L) out.bucket_off[L] = 0;
    if (n == 0) return TCRNET_OK;
    const int nblocks = (int)ceil_div(n, kPackThreads);
    if (keep_input_order) {
        TCR_CHECK(out.canon_in.alloc_owned(sizeof(Canon) * n, s));  // kept by the handle
        TCR_CHECK(out.lens.alloc_owned(n, s));
    } else {
        TCR_CHECK(out.canon_in.alloc(sizeof(Canon) * n, s));
        TCR_CHECK(out.lens.alloc(n, s));
    }
    if (bucket) {
        TCR_CHECK(out.canon.alloc_owned(sizeof(Canon) * n, s));  // kept by the handle
        TCR_CHECK(out.perm.alloc_owned(sizeof(int32_t) * n, s));
    }
    const int64_t ncnt = (int64_t)kBins * nblocks;
    DevBuf blockcnt, blockoff, bounds;
    if (bucket) {
        TCR_CHECK(blockcnt.alloc(sizeof(int32_t) * ncnt, s));
        TCR_CHECK(blockoff.alloc(sizeof(int64_t) * (ncnt + 1), s));
        TCR_CHECK(bounds.alloc(sizeof(int64_t) * (kBins + 1), s));
    }
    TCR_CHECK(out.flags.alloc(sizeof(unsigned long long) * 2, s));  // [0] first error, [1] total length
    unsigned long long* d_flags = out.flags.as<unsigned long long>();
    TCR_CUDA(cudaMemsetAsync(d_flags, 0, 2 * sizeof(unsigned long long), s));
    k_encode<<<nblocks, kPackThreads, 0, s>>>(d_chars, d_offsets, n, lo, hi, out.canon_in.as<Canon>(),
                                              out.lens.as<uint8_t>(), bucket ? blockcnt.as<int32_t>() : nullptr,
                                              nblocks, d_flags, d_flags + 1);
    TCR_LAUNCH_CHECK();
    if (defer_check && !bucket) {
        out.lensum = -1;
        return TCRNET_OK;
    }
    unsigned long long h_flags[2] = {0, 0};
    TCR_CUDA(cudaMemcpyAsync(h_flags, d_flags, sizeof(h_flags), cudaMemcpyDeviceToHost, s));
    int64_t h_bounds[kBins + 1];
    if (bucket) {
        TCR_CHECK(scan_exclusive_i32_to_i64(blockcnt.as<int32_t>(), blockoff.as<int64_t>(), ncnt, s));
        k_bucket_bounds<<<1, 64, 0, s>>>(blockoff.as<int64_t>(), nblocks, bounds.as<int64_t>());
        TCR_LAUNCH_CHECK();
        TCR_CUDA(cudaMemcpyAsync(h_bounds, bounds.as<void>(), sizeof(h_bounds), cudaMemcpyDeviceToHost, s));
    }
    TCR_CUDA(cudaStreamSynchronize(s));
    TCR_CHECK(pack_flags_status(h_flags[0], bad_index));
    out.lensum = (int64_t)h_flags[1];
    if (!bucket) return TCRNET_OK;
    for (int L = 0; L <= kBins; ++L) out.bucket_off[L] = h_bounds[L];
    k_bucket_scatter<<<nblocks, kPackThreads, 0, s>>>(out.canon_in.as<Canon>(), out.lens.as<uint8_t>(), n,
                                                      blockoff.as<int64_t>(), nblocks, out.canon.as<Canon>(),
                                                      out.perm.as<int32_t>());
    TCR_LAUNCH_CHECK();
    return TCRNET_OK;
}

}  // namespace tcr
