// Plain and sizing kernels for ORC RLE v1 and v2: one CTA per chunk, one
// part of the chunk per warp.
#include "chunk.cuh"

namespace codag {

__global__ void __launch_bounds__(512) rle_v1_kernel(Args a) { rle_cta_body<1, true>(a, a.stage_bytes); }
__global__ void __launch_bounds__(512) rle_v1_sizes_kernel(Args a) {
  rle_cta_body<1, false>(a, a.stage_bytes);
}
__global__ void __launch_bounds__(512) rle_v2_kernel(Args a) { rle_cta_body<2, true>(a, a.stage_bytes); }
// ORC byte / boolean RLE as a plain call: a CTA per chunk, like the above
__global__ void __launch_bounds__(512) byte_rle_cta_kernel(Args a) { rle_cta_body<4, true>(a, a.stage_bytes); }
__global__ void __launch_bounds__(512) rle_v2_sizes_kernel(Args a) {
  rle_cta_body<2, false>(a, a.stage_bytes);
}
__global__ void __launch_bounds__(kThreads) rle_v2_walk_kernel(Args a) { rle_v2_walk_body(a); }

// this unit's copy of the work-wait bound (codag_set_wait_limit_ns)
cudaError_t set_wait_limit_rle(uint64_t ns) { return set_wait_limit_here(ns); }

}  // namespace codag
