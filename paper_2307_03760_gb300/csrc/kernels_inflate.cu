// Plain and sizing kernels for raw Deflate: one warp per chunk.
#include "chunk.cuh"

namespace codag {

__global__ void __launch_bounds__(kThreads) inflate_kernel(Args a) {
  chunk_body<3, true, kDeflateWarp, DeflateRing>(a);
}
__global__ void __launch_bounds__(kThreads) inflate_sizes_kernel(Args a) {
  chunk_body<3, false, kDeflateWarp, DeflateRing>(a);
}

}  // namespace codag
