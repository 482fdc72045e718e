// Integer-issue microbenchmark (measurement aid, no counterpart in the paper).
//
// The all-pairs tile kernel is bound by integer instruction issue, so its
// roofline needs the chip's integer rate per SM and clock. This kernel measures
// it: every thread runs independent chains of one kind of 32-bit integer
// instruction (three-input logic LOP3, funnel shift SHF, add, multiply-add
// IMAD, population count POPC, or a mix of LOP3 + add + IMAD that spreads over
// the ALU and FMA pipes), and the caller times the launch with CUDA events.
// Each chain step reads the two values updated just before
// it (a rotating triple), so the compiler can neither merge steps into one
// instruction nor drop them; eight triples per thread give enough independent
// work to keep the pipes busy. Every thread writes one word of the output (the
// combined chains), so the work is live and all stores stay in bounds.
#include "common.cuh"

namespace tcr {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;  // independent triples per thread

__device__ __forceinline__ uint32_t lop3_xor3(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

__device__ __forceinline__ uint32_t shf_l(uint32_t lo, uint32_t hi, uint32_t s) {
    uint32_t d;
    asm volatile("shf.l.wrap.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(lo), "r"(hi), "r"(s));
    return d;
}

__device__ __forceinline__ uint32_t add2(uint32_t a, uint32_t b) {
    uint32_t d;
    asm volatile("add.u32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

__device__ __forceinline__ uint32_t mad(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm volatile("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

__device__ __forceinline__ uint32_t popc_add(uint32_t a, uint32_t b) {
    uint32_t d;
    asm volatile("popc.b32 %0, %1;" : "=r"(d) : "r"(a ^ b));
    return d;
}

// One step of kind K on triple (x, y, z) (ops_per_step(K) instructions).
template <int K>
__device__ __forceinline__ void step(uint32_t& x, uint32_t& y, uint32_t& z, uint32_t s) {
    if constexpr (K == TCRNET_PROBE_LOP3) {
        x = lop3_xor3(x, y, z);
        y = lop3_xor3(y, z, x);
        z = lop3_xor3(z, x, y);
    } else if constexpr (K == TCRNET_PROBE_SHF) {
        x = shf_l(x, y, s);
        y = shf_l(y, z, s);
        z = shf_l(z, x, s);
    } else if constexpr (K == TCRNET_PROBE_IADD) {
        x = add2(x, y);
        y = add2(y, z);
        z = add2(z, x);
    } else if constexpr (K == TCRNET_PROBE_IMAD) {
        x = mad(x, y, z);
        y = mad(y, z, x);
        z = mad(z, x, y);
    } else if constexpr (K == TCRNET_PROBE_POPC) {
        x = popc_add(x, y) + z;
        y = popc_add(y, z) + x;
        z = popc_add(z, x) + y;
    } else {  // mix: one LOP3, one add, one IMAD per step
        x = lop3_xor3(x, y, z);
        y = add2(y, x);
        z = mad(z, x, y);
    }
}

template <int K>
__global__ void __launch_bounds__(kProbeThreads) k_int_probe(uint32_t* __restrict__ out, int64_t n_threads,
                                                             int iters, uint32_t seed) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_threads) return;
    uint32_t x[kChains], y[kChains], z[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        x[c] = seed ^ (uint32_t)(t * 2654435761u) ^ (uint32_t)c;
        y[c] = x[c] * 0x9e3779b9u + 1u;
        z[c] = y[c] ^ 0x85ebca6bu;
    }
    const uint32_t s = 1u + (seed & 7u);
#pragma unroll 4  // loop control stays a few percent of the issued instructions
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) step<K>(x[c], y[c], z[c], s);
    }
    uint32_t acc = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc ^= x[c] ^ y[c] ^ z[c];
    out[t] = acc;
}

// Integer instructions one step issues per thread, per kind (a POPC sub-step
// issues the xor, the POPC and an add).
int ops_per_step(int kind) {
    switch (kind) {
        case TCRNET_PROBE_POPC: return 3 * 3;
        default: return 3;
    }
}

}  // namespace
}  // namespace tcr

extern "C" tcrnet_status tcrnet_probe_int_issue(int32_t kind, int32_t iters, uint32_t* d_out, int64_t n_threads,
                                                void* stream, int64_t* ops_per_thread) {
    using namespace tcr;
    if (ops_per_thread) *ops_per_thread = 0;
    if (!d_out || iters < 1 || n_threads < 1 || n_threads % kProbeThreads != 0 ||
        n_threads / kProbeThreads > 0x7fffffffLL || kind < TCRNET_PROBE_LOP3 || kind > TCRNET_PROBE_MIX)
        return TCRNET_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned grid = (unsigned)(n_threads / kProbeThreads);
    const uint32_t seed = 0x2112u;
    switch (kind) {
        case TCRNET_PROBE_LOP3:
            k_int_probe<TCRNET_PROBE_LOP3><<<grid, kProbeThreads, 0, s>>>(d_out, n_threads, iters, seed);
            break;
        case TCRNET_PROBE_SHF:
            k_int_probe<TCRNET_PROBE_SHF><<<grid, kProbeThreads, 0, s>>>(d_out, n_threads, iters, seed);
            break;
        case TCRNET_PROBE_IADD:
            k_int_probe<TCRNET_PROBE_IADD><<<grid, kProbeThreads, 0, s>>>(d_out, n_threads, iters, seed);
            break;
        case TCRNET_PROBE_IMAD:
            k_int_probe<TCRNET_PROBE_IMAD><<<grid, kProbeThreads, 0, s>>>(d_out, n_threads, iters, seed);
            break;
        case TCRNET_PROBE_POPC:
            k_int_probe<TCRNET_PROBE_POPC><<<grid, kProbeThreads, 0, s>>>(d_out, n_threads, iters, seed);
            break;
        default:
            k_int_probe<TCRNET_PROBE_MIX><<<grid, kProbeThreads, 0, s>>>(d_out, n_threads, iters, seed);
            break;
    }
    TCR_CUDA(cudaGetLastError());
    note_launch();
    if (ops_per_thread) *ops_per_thread = (int64_t)iters * kChains * ops_per_step(kind);
    return TCRNET_OK;
}
