// Two-pass raw Deflate: the Huffman pass (one lane per chunk) and the LZ77
// copy pass (one warp per chunk).  Bodies in inflate_lanes.cuh.
#include "chunk.cuh"
#include "inflate_lanes.cuh"

namespace codag {

__global__ void __launch_bounds__(32 * kHufWarps, 1) inflate_huffman_kernel(Args a, HufArgs h) {
  huffman_body<true>(a, h);
}
__global__ void __launch_bounds__(32 * kHufWarps, 1) inflate_huffman_sizes_kernel(Args a, HufArgs h) {
  huffman_body<false>(a, h);
}
__global__ void __launch_bounds__(32 * kLz77Warps) inflate_lz77_kernel(Args a, HufArgs h) {
  const uint64_t c = (uint64_t)blockIdx.x * kLz77Warps + (threadIdx.x >> 5);
  if (c < a.n) lz77_chunk(a, h, c);
}

}  // namespace codag
