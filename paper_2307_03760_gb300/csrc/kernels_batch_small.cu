// Batch kernel instances with small input-ring slots (2 KiB and 4 KiB rings).
#include "batch.cuh"

namespace codag {

CODAG_BATCH_SHAPE(256, 8)
CODAG_BATCH_SHAPE(512, 8)

// this unit's copy of the work-wait bound (codag_set_wait_limit_ns)
cudaError_t set_wait_limit_batch_small(uint64_t ns) { return set_wait_limit_here(ns); }

}  // namespace codag
