// Network analytics on the device CSR (the analyses of the paper's Results that
// consume the network): connected components under node removal (Methods
// "Computing LCC": the largest connected component, LCC(p) after removing a
// fraction p of the nodes) and the average neighbour degree d_nn (Methods
// "Overview of network theory concepts").
//
// Components: lock-free union-find over the undirected edges {i, j}, i < j,
// both kept. A union links the larger root below the smaller one (compare-and-
// swap on the root's parent, retried when another thread moved it), so every
// parent pointer only decreases and points to a node of the same set; `find`
// walks strictly decreasing ids (terminates) and halves the path as it goes.
// Each final root is the smallest node id of its component, which makes the
// labels deterministic. Component sizes by atomic counting; the number of
// components and the largest size by a grid reduction.
#include <algorithm>

#include "kernels.cuh"

namespace tcr {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kDefaultLinkAttempts = 1 << 20;

__device__ __forceinline__ int32_t find_root(int32_t* parent, int32_t x) {
    volatile int32_t* vp = parent;
    int32_t p = vp[x];
    while (p != x) {
        const int32_t gp = vp[p];
        if (gp != p) vp[x] = gp;  // path halving (benign: gp is an ancestor of x)
        x = p;
        p = gp;
    }
    return x;
}

__global__ void k_cc_init(const uint8_t* __restrict__ keep, int64_t n, int32_t* __restrict__ parent,
                          int32_t* __restrict__ size) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    parent[i] = (keep == nullptr || keep[i]) ? (int32_t)i : -1;
    size[i] = 0;
}

template <typename Off>
__global__ void __launch_bounds__(kThreads)
k_cc_link(const Off* __restrict__ off, const int32_t* __restrict__ cols, int64_t n, int32_t* parent,
          int max_attempts, int* __restrict__ err) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += stride) {
        if (parent[i] < 0) continue;  // removed (set before this kernel; uniform per warp)
        const int64_t b = off[i], e = off[i + 1];
        for (int64_t k = b + lane; k < e; k += 32) {
            const int32_t j = cols[k];
            if (j <= i || ((volatile int32_t*)parent)[j] < 0) continue;
            int32_t a = (int32_t)i, c = j;
            int it = 0;
            for (; it < max_attempts; ++it) {
                int32_t ra = find_root(parent, a), rc = find_root(parent, c);
                if (ra == rc) break;
                if (ra > rc) {
                    const int32_t t = ra;
                    ra = rc;
                    rc = t;
                }
                if (atomicCAS(&parent[rc], rc, ra) == rc) break;
                a = ra;
                c = rc;
            }
            if (it == max_attempts) atomicExch(err, 1);  // gave up on this edge; the host reports it
        }
    }
}

__global__ void k_cc_label(int64_t n, int32_t* parent, int32_t* __restrict__ labels, int32_t* __restrict__ size) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (parent[i] < 0) {
        labels[i] = -1;
        return;
    }
    const int32_t r = find_root(parent, (int32_t)i);
    labels[i] = r;
    atomicAdd(&size[r], 1);
}

__global__ void k_cc_reduce(int64_t n, const int32_t* __restrict__ labels, const int32_t* __restrict__ size,
                            unsigned long long* __restrict__ out /* [0] components, [1] largest */) {
    unsigned long long roots = 0, largest = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (labels[i] == (int32_t)i) {
            ++roots;
            largest = largest > (unsigned long long)size[i] ? largest : (unsigned long long)size[i];
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        roots += __shfl_down_sync(kFull, roots, d);
        const unsigned long long o = __shfl_down_sync(kFull, largest, d);
        largest = largest > o ? largest : o;
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&out[0], roots);
        atomicMax(&out[1], largest);
    }
}

template <typename Off>
__global__ void __launch_bounds__(kThreads)
k_neighbor_degree(const Off* __restrict__ off, const int32_t* __restrict__ cols, int64_t n,
                  double* __restrict__ knn) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += stride) {
        const int64_t b = off[i], e = off[i + 1];
        long long s = 0;
        for (int64_t k = b + lane; k < e; k += 32) {
            const int32_t j = cols[k];
            s += (long long)(off[j + 1] - off[j]);
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) s += __shfl_down_sync(kFull, s, d);
        if (lane == 0) knn[i] = (e > b) ? (double)s / (double)(e - b) : 0.0;
    }
}

// Degree histogram: bins in shared memory per block when they fit, global
// atomics otherwise; the last bin collects every larger degree.
constexpr int kSmemBins = 4096;

__global__ void __launch_bounds__(kThreads)
k_degree_hist(const int32_t* __restrict__ deg, int64_t n, unsigned long long* __restrict__ hist, int64_t nbins,
              int* __restrict__ dmax) {
    __shared__ unsigned int bins[kSmemBins];
    const bool local = nbins <= kSmemBins;
    if (local)
        for (int b = threadIdx.x; b < nbins; b += blockDim.x) bins[b] = 0;
    __syncthreads();
    int mymax = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int d = deg[i];
        mymax = d > mymax ? d : mymax;
        const int64_t b = (int64_t)d < nbins - 1 ? (int64_t)d : nbins - 1;
        if (local) atomicAdd(&bins[b], 1u);
        else atomicAdd(&hist[b], 1ull);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const int t = __shfl_down_sync(kFull, mymax, o);
        mymax = t > mymax ? t : mymax;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(dmax, mymax);
    __syncthreads();
    if (local)
        for (int b = threadIdx.x; b < nbins; b += blockDim.x)
            if (bins[b]) atomicAdd(&hist[b], (unsigned long long)bins[b]);
}

// ---- the same analyses on the graph of distinct strings --------------------
// A deletion build keeps node -> distinct string (uid) and the edges between
// distinct strings, each once. The members of a distinct string are a clique,
// so with node removal a string is present iff one of its members is kept,
// the network's components are those of the string graph restricted to
// present strings, and a kept node's component is its string's. Work is
// proportional to the U strings and E edges instead of the nnz entries.

__global__ void k_dcc_init(const int32_t* __restrict__ uid, const uint8_t* __restrict__ keep, int64_t n,
                           int32_t* __restrict__ present) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && (keep == nullptr || keep[i])) present[uid[i]] = 1;
}

__global__ void k_dcc_parent(const int32_t* __restrict__ present, int64_t U, int32_t* __restrict__ parent,
                             int32_t* __restrict__ cmin, int32_t* __restrict__ size) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= U) return;
    parent[u] = present[u] ? (int32_t)u : -1;
    cmin[u] = 0x7fffffff;
    size[u] = 0;
}

__global__ void k_dcc_link(const int2* __restrict__ edges, int64_t E, int32_t* parent, int max_attempts,
                           int* __restrict__ err) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < E; k += (int64_t)gridDim.x * blockDim.x) {
        const int2 e = edges[k];
        if (((volatile int32_t*)parent)[e.x] < 0 || ((volatile int32_t*)parent)[e.y] < 0) continue;
        int32_t a = e.x, c = e.y;
        int it = 0;
        for (; it < max_attempts; ++it) {
            int32_t ra = find_root(parent, a), rc = find_root(parent, c);
            if (ra == rc) break;
            if (ra > rc) {
                const int32_t t = ra;
                ra = rc;
                rc = t;
            }
            if (atomicCAS(&parent[rc], rc, ra) == rc) break;
            a = ra;
            c = rc;
        }
        if (it == max_attempts) atomicExch(err, 1);  // gave up on this edge; the host reports it
    }
}

// every present string points at its root afterwards (one find per string)
__global__ void k_dcc_flatten(int64_t U, int32_t* parent, int32_t* __restrict__ root) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= U) return;
    root[u] = parent[u] < 0 ? -1 : find_root(parent, (int32_t)u);
}

// per kept node: its string's root collects the smallest kept node id and the
// size. Lanes of a warp with the same root combine first (the largest
// component's root would otherwise take one atomic per member).
__global__ void k_dcc_members(const int32_t* __restrict__ uid, const uint8_t* __restrict__ keep, int64_t n,
                              const int32_t* __restrict__ root, int32_t* __restrict__ cmin,
                              int32_t* __restrict__ size) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool kept = i < n && (keep == nullptr || keep[i]);
    const int32_t r = kept ? root[uid[i]] : -1;
    const unsigned peers = __match_any_sync(kFull, r);
    if (!kept) return;
    const int lane = threadIdx.x & 31;
    // node ids grow with the lane, so the lowest peer holds the smallest id
    const int leader = __ffs(peers) - 1;
    if (lane == leader) {
        atomicMin(&cmin[r], (int32_t)i);
        atomicAdd(&size[r], __popc(peers));
    }
}

__global__ void k_dcc_label(const int32_t* __restrict__ uid, const uint8_t* __restrict__ keep, int64_t n,
                            const int32_t* __restrict__ root, const int32_t* __restrict__ cmin,
                            int32_t* __restrict__ labels) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    labels[i] = (keep != nullptr && !keep[i]) ? -1 : cmin[root[uid[i]]];
}

__global__ void k_dcc_reduce(const int32_t* __restrict__ parent, const int32_t* __restrict__ size, int64_t U,
                             unsigned long long* __restrict__ out /* [0] components, [1] largest */) {
    unsigned long long roots = 0, largest = 0;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < U; u += (int64_t)gridDim.x * blockDim.x) {
        if (parent[u] == (int32_t)u) {
            ++roots;
            largest = largest > (unsigned long long)size[u] ? largest : (unsigned long long)size[u];
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        roots += __shfl_down_sync(kFull, roots, d);
        const unsigned long long o = __shfl_down_sync(kFull, largest, d);
        largest = largest > o ? largest : o;
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&out[0], roots);
        atomicMax(&out[1], largest);
    }
}

// d_nn per distinct string u: the members of u other than i (m_u - 1 nodes of
// degree D_u - 1) and the members of each neighbour string v (m_v nodes of
// degree D_v - 1), over the degree D_u - 1 of each member of u.
__global__ void k_dknn_self(const int32_t* __restrict__ umult, const int64_t* __restrict__ dsize, int64_t U,
                            double* __restrict__ acc) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u < U) acc[u] = (double)(umult[u] - 1) * (double)(dsize[u] - 1);
}

__global__ void k_dknn_edges(const int2* __restrict__ edges, int64_t E, const int32_t* __restrict__ umult,
                             const int64_t* __restrict__ dsize, double* __restrict__ acc) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < E; k += (int64_t)gridDim.x * blockDim.x) {
        const int2 e = edges[k];
        atomicAdd(&acc[e.x], (double)umult[e.y] * (double)(dsize[e.y] - 1));
        atomicAdd(&acc[e.y], (double)umult[e.x] * (double)(dsize[e.x] - 1));
    }
}

__global__ void k_dsize_edges(const int2* __restrict__ edges, int64_t E, const int32_t* __restrict__ umult,
                              unsigned long long* __restrict__ dsize) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < E; k += (int64_t)gridDim.x * blockDim.x) {
        const int2 e = edges[k];
        atomicAdd(&dsize[e.x], (unsigned long long)umult[e.y]);
        atomicAdd(&dsize[e.y], (unsigned long long)umult[e.x]);
    }
}

__global__ void k_dsize_self(const int32_t* __restrict__ umult, int64_t U, unsigned long long* __restrict__ dsize) {
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u < U) dsize[u] = (unsigned long long)umult[u];
}

__global__ void k_dknn_nodes(const int32_t* __restrict__ uid, int64_t n, const int64_t* __restrict__ dsize,
                             const double* __restrict__ acc, double* __restrict__ knn) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t u = uid[i];
    const int64_t d = dsize[u] - 1;
    knn[i] = d > 0 ? acc[u] / (double)d : 0.0;
}

inline unsigned blocks_for(int64_t n, int per_block, int num_sms) {
    const int64_t b = ceil_div(n, per_block);
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)num_sms * 32));
}

}  // namespace

tcrnet_status components(const void* off, bool off64, const int32_t* cols, int64_t n, const uint8_t* keep,
                         int32_t* labels, int64_t* n_components, int64_t* largest, cudaStream_t s, int num_sms,
                         int link_attempts) {
    const int attempts = link_attempts > 0 ? link_attempts : kDefaultLinkAttempts;
    *n_components = 0;
    *largest = 0;
    if (n == 0) return TCRNET_OK;
    DevBuf parent, size, red;
    TCR_CHECK(parent.alloc(sizeof(int32_t) * n, s));
    TCR_CHECK(size.alloc(sizeof(int32_t) * n, s));
    TCR_CHECK(red.alloc(sizeof(unsigned long long) * 2 + sizeof(int), s));
    TCR_CUDA(cudaMemsetAsync(red.as<void>(), 0, sizeof(unsigned long long) * 2 + sizeof(int), s));
    int* err = reinterpret_cast<int*>(red.as<unsigned long long>() + 2);
    k_cc_init<<<(unsigned)ceil_div(n, kThreads), kThreads, 0, s>>>(keep, n, parent.as<int32_t>(), size.as<int32_t>());
    TCR_LAUNCH_CHECK();
    const unsigned wb = blocks_for(n, kWarps, num_sms);
    if (off64)
        k_cc_link<int64_t><<<wb, kThreads, 0, s>>>(static_cast<const int64_t*>(off), cols, n, parent.as<int32_t>(),
                                                   attempts, err);
    else
        k_cc_link<int32_t><<<wb, kThreads, 0, s>>>(static_cast<const int32_t*>(off), cols, n, parent.as<int32_t>(),
                                                   attempts, err);
    TCR_LAUNCH_CHECK();
    k_cc_label<<<(unsigned)ceil_div(n, kThreads), kThreads, 0, s>>>(n, parent.as<int32_t>(), labels, size.as<int32_t>());
    TCR_LAUNCH_CHECK();
    k_cc_reduce<<<blocks_for(n, kThreads, num_sms), kThreads, 0, s>>>(n, labels, size.as<int32_t>(),
                                                                       red.as<unsigned long long>());
    TCR_LAUNCH_CHECK();
    unsigned long long h[2] = {0, 0};
    int h_err = 0;
    TCR_CUDA(cudaMemcpyAsync(h, red.as<void>(), sizeof(h), cudaMemcpyDeviceToHost, s));
    TCR_CUDA(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    TCR_CUDA(cudaStreamSynchronize(s));
    if (h_err) return TCRNET_ETIMEOUT;
    *n_components = (int64_t)h[0];
    *largest = (int64_t)h[1];
    return TCRNET_OK;
}

tcrnet_status components_distinct(const int32_t* uid, int64_t n, const int2* edges, int64_t E, int64_t U,
                                  const uint8_t* keep, int32_t* labels, int64_t* n_components, int64_t* largest,
                                  cudaStream_t s, int num_sms, int link_attempts) {
    const int attempts = link_attempts > 0 ? link_attempts : kDefaultLinkAttempts;
    *n_components = 0;
    *largest = 0;
    if (n == 0) return TCRNET_OK;
    DevBuf present, parent, cmin, size, red, root;
    TCR_CHECK(present.alloc(sizeof(int32_t) * U, s));
    TCR_CHECK(root.alloc(sizeof(int32_t) * U, s));
    TCR_CHECK(parent.alloc(sizeof(int32_t) * U, s));
    TCR_CHECK(cmin.alloc(sizeof(int32_t) * U, s));
    TCR_CHECK(size.alloc(sizeof(int32_t) * U, s));
    TCR_CHECK(red.alloc(sizeof(unsigned long long) * 2 + sizeof(int), s));
    TCR_CUDA(cudaMemsetAsync(present.as<void>(), 0, sizeof(int32_t) * U, s));
    TCR_CUDA(cudaMemsetAsync(red.as<void>(), 0, sizeof(unsigned long long) * 2 + sizeof(int), s));
    int* err = reinterpret_cast<int*>(red.as<unsigned long long>() + 2);
    const unsigned gn = (unsigned)ceil_div(n, kThreads), gu = (unsigned)ceil_div(U, kThreads);
    k_dcc_init<<<gn, kThreads, 0, s>>>(uid, keep, n, present.as<int32_t>());
    TCR_LAUNCH_CHECK();
    k_dcc_parent<<<gu, kThreads, 0, s>>>(present.as<int32_t>(), U, parent.as<int32_t>(), cmin.as<int32_t>(),
                                         size.as<int32_t>());
    TCR_LAUNCH_CHECK();
    if (E > 0) {
        k_dcc_link<<<blocks_for(E, kThreads, num_sms), kThreads, 0, s>>>(edges, E, parent.as<int32_t>(), attempts,
                                                                         err);
        TCR_LAUNCH_CHECK();
    }
    k_dcc_flatten<<<gu, kThreads, 0, s>>>(U, parent.as<int32_t>(), root.as<int32_t>());
    TCR_LAUNCH_CHECK();
    k_dcc_members<<<gn, kThreads, 0, s>>>(uid, keep, n, root.as<int32_t>(), cmin.as<int32_t>(), size.as<int32_t>());
    TCR_LAUNCH_CHECK();
    if (labels) {
        k_dcc_label<<<gn, kThreads, 0, s>>>(uid, keep, n, root.as<int32_t>(), cmin.as<int32_t>(), labels);
        TCR_LAUNCH_CHECK();
    }
    k_dcc_reduce<<<blocks_for(U, kThreads, num_sms), kThreads, 0, s>>>(parent.as<int32_t>(), size.as<int32_t>(), U,
                                                                       red.as<unsigned long long>());
    TCR_LAUNCH_CHECK();
    unsigned long long h[2] = {0, 0};
    int h_err = 0;
    TCR_CUDA(cudaMemcpyAsync(h, red.as<void>(), sizeof(h), cudaMemcpyDeviceToHost, s));
    TCR_CUDA(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    TCR_CUDA(cudaStreamSynchronize(s));
    if (h_err) return TCRNET_ETIMEOUT;
    *n_components = (int64_t)h[0];
    *largest = (int64_t)h[1];
    return TCRNET_OK;
}

tcrnet_status neighbor_degree_distinct(const int32_t* uid, int64_t n, const int2* edges, int64_t E,
                                       const int32_t* umult, int64_t U, double* knn, cudaStream_t s, int num_sms) {
    if (n == 0) return TCRNET_OK;
    DevBuf dsize, acc;
    TCR_CHECK(dsize.alloc(sizeof(int64_t) * U, s));
    TCR_CHECK(acc.alloc(sizeof(double) * U, s));
    const unsigned gu = (unsigned)ceil_div(U, kThreads);
    auto* ds = reinterpret_cast<unsigned long long*>(dsize.as<int64_t>());
    k_dsize_self<<<gu, kThreads, 0, s>>>(umult, U, ds);
    TCR_LAUNCH_CHECK();
    if (E > 0) {
        k_dsize_edges<<<blocks_for(E, kThreads, num_sms), kThreads, 0, s>>>(edges, E, umult, ds);
        TCR_LAUNCH_CHECK();
    }
    k_dknn_self<<<gu, kThreads, 0, s>>>(umult, dsize.as<int64_t>(), U, acc.as<double>());
    TCR_LAUNCH_CHECK();
    if (E > 0) {
        k_dknn_edges<<<blocks_for(E, kThreads, num_sms), kThreads, 0, s>>>(edges, E, umult, dsize.as<int64_t>(),
                                                                           acc.as<double>());
        TCR_LAUNCH_CHECK();
    }
    k_dknn_nodes<<<(unsigned)ceil_div(n, kThreads), kThreads, 0, s>>>(uid, n, dsize.as<int64_t>(), acc.as<double>(),
                                                                     knn);
    TCR_LAUNCH_CHECK();
    return TCRNET_OK;
}

tcrnet_status neighbor_degree(const void* off, bool off64, const int32_t* cols, int64_t n, double* knn,
                              cudaStream_t s, int num_sms) {
    if (n == 0) return TCRNET_OK;
    const unsigned wb = blocks_for(n, kWarps, num_sms);
    if (off64)
        k_neighbor_degree<int64_t><<<wb, kThreads, 0, s>>>(static_cast<const int64_t*>(off), cols, n, knn);
    else
        k_neighbor_degree<int32_t><<<wb, kThreads, 0, s>>>(static_cast<const int32_t*>(off), cols, n, knn);
    TCR_LAUNCH_CHECK();
    return TCRNET_OK;
}

tcrnet_status degree_histogram(const int32_t* deg, int64_t n, int64_t* hist, int64_t nbins, int64_t* max_degree,
                               cudaStream_t s, int num_sms) {
    DevBuf dm;
    TCR_CHECK(dm.alloc(sizeof(int), s));
    TCR_CUDA(cudaMemsetAsync(dm.as<void>(), 0, sizeof(int), s));
    TCR_CUDA(cudaMemsetAsync(hist, 0, sizeof(int64_t) * nbins, s));
    if (n > 0) {
        const unsigned grid = std::min(blocks_for(n, kThreads, num_sms), (unsigned)num_sms * 2);
        k_degree_hist<<<grid, kThreads, 0, s>>>(deg, n, reinterpret_cast<unsigned long long*>(hist), nbins,
                                                dm.as<int>());
        TCR_LAUNCH_CHECK();
    }
    int h_max = 0;
    TCR_CUDA(cudaMemcpyAsync(&h_max, dm.as<int>(), sizeof(int), cudaMemcpyDeviceToHost, s));
    TCR_CUDA(cudaStreamSynchronize(s));
    if (max_degree) *max_degree = h_max;
    return TCRNET_OK;
}

}  // namespace tcr
