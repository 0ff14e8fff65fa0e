// Plain and sizing kernels for ORC RLE v1 and v2: one warp per chunk.
#include "chunk.cuh"

namespace codag {

__global__ void __launch_bounds__(kThreads) rle_v1_kernel(Args a) {
  chunk_body<1, true, kRleV1Warp, RleRing>(a);
}
__global__ void __launch_bounds__(kThreads) rle_v1_sizes_kernel(Args a) {
  chunk_body<1, false, kRleV1Warp, RleRing>(a);
}
__global__ void __launch_bounds__(kThreads) rle_v2_kernel(Args a) {
  chunk_body<2, true, kRleV2Warp, RleRing>(a);
}
__global__ void __launch_bounds__(kThreads) rle_v2_sizes_kernel(Args a) {
  chunk_body<2, false, kRleV2Warp, RleRing>(a);
}

}  // namespace codag
