// Plain and sizing kernels with one warp per chunk: raw Deflate, ORC zlib
// streams, ORC byte / boolean RLE.
#include "chunk.cuh"

namespace codag {

__global__ void __launch_bounds__(kThreads, 10) inflate_kernel(Args a) { warp_chunk_body<3, true>(a); }
__global__ void __launch_bounds__(kThreads) inflate_sizes_kernel(Args a) {
  warp_chunk_body<3, false>(a);
}
// ORC zlib streams: 7 CTAs per SM (72 registers, 24 bytes of spills against
// 88 at 10 CTAs) is 15% faster on the 1 GiB column of 4,096 streams, which
// are then all resident at once
__global__ void __launch_bounds__(kThreads, 7) orc_zlib_kernel(Args a) { warp_chunk_body<5, true>(a); }
__global__ void __launch_bounds__(kThreads) orc_zlib_sizes_kernel(Args a) {
  warp_chunk_body<5, false>(a);
}
// byte RLE consumes its input about ten times faster per instruction than
// Deflate: it stages through the 4 KiB ring, so that refills run well ahead
__global__ void __launch_bounds__(kThreads) byte_rle_kernel(Args a) { warp_chunk_body<4, true, RleRing>(a); }
// the same decoders with the register staging ring (no shared-memory input)
__global__ void __launch_bounds__(kThreads, 10) inflate_reg_kernel(Args a) {
  warp_chunk_body<3, true, RegRing>(a);
}
__global__ void __launch_bounds__(kThreads) byte_rle_reg_kernel(Args a) {
  warp_chunk_body<4, true, RegRing>(a);
}
__global__ void __launch_bounds__(kThreads) byte_rle_sizes_kernel(Args a) {
  warp_chunk_body<4, false, RleRing>(a);
}

// this unit's copy of the work-wait bound (codag_set_wait_limit_ns)
cudaError_t set_wait_limit_inflate(uint64_t ns) { return set_wait_limit_here(ns); }

}  // namespace codag
