// Deletion-neighbourhood method (hot-path step a7): declarations.
#pragma once

#include "kernels.cuh"

namespace tcr {

// AUTO picks the deletion method from this many strings on.
constexpr int64_t kAutoDeletionMinN = 1LL << 62;

struct DeletionResult {
    DevBuf off64;   // int64[n + 1]
    DevBuf cols;    // int32[nnz]
    DevBuf degree;  // int32[n]
    int64_t nnz = 0;
    int64_t n_unique = 0;
    int64_t n_records = 0;
    int64_t unique_edges = 0;
    double ms_join = 0, ms_scan = 0, ms_fill = 0, ms_sort = 0;
    double ms_phase[8] = {0};
};

tcrnet_status deletion_build(const Packed& pk, int T, DeletionResult& out, cudaStream_t s, int num_sms,
                             bool profile);

}  // namespace tcr
