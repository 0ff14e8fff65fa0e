// Batch kernel instance with 2 KiB input-ring slots (an 8 KiB ring per warp).
#include "batch.cuh"

namespace codag {

CODAG_BATCH_SHAPE(2048, 4)

// this unit's copy of the work-wait bound (codag_set_wait_limit_ns)
cudaError_t set_wait_limit_batch_large(uint64_t ns) { return set_wait_limit_here(ns); }

}  // namespace codag
