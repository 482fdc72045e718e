#include "deletion.cuh"

namespace tcr {
tcrnet_status deletion_build(const Packed&, int, DeletionResult&, cudaStream_t, int, bool) { return TCRNET_ENOTSUP; }
}  // namespace tcr
