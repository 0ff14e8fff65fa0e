// Plain and sizing kernels for raw Deflate: one warp per chunk.
#include "chunk.cuh"

namespace codag {

__global__ void __launch_bounds__(kThreads, 10) inflate_kernel(Args a) { inflate_warp_body<true>(a); }
__global__ void __launch_bounds__(kThreads) inflate_sizes_kernel(Args a) {
  inflate_warp_body<false>(a);
}

}  // namespace codag
