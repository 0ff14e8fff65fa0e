// Kernel entry points and their per-warp shared-memory layouts.
//
// Work mapping (CODAG Sec. II-B and V-C): every chunk is independent; one
// warp decodes one chunk.  The plain kernels launch one warp per chunk and
// let the block scheduler hand out chunks; the batch kernel is persistent
// (one wave of CTAs) and its warps claim chunks with an atomic counter in
// descending-size order, so a mixed batch of uneven chunks keeps every SM busy
// and the largest chunks start first.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "inflate.cuh"
#include "rle_v1.cuh"
#include "rle_v2.cuh"

namespace codag {

constexpr int kWarpsPerBlock = 4;
constexpr int kThreads = 32 * kWarpsPerBlock;

using RleRing = InRing<1024, 4>;
using DeflateRing = InRing<512, 4>;
constexpr int kLitTB = 10, kDistTB = 8, kWin = 4096;
using DeflateSmem = InflateSmem<kLitTB, kDistTB, kWin>;

constexpr int round128(int x) { return (x + 127) & ~127; }
constexpr int cmax(int a, int b) { return a > b ? a : b; }

constexpr int kRleV1Warp = round128(RleRing::SMEM + kRleV1Scratch);
constexpr int kRleV2Warp = round128(RleRing::SMEM + kRleV2Scratch);
constexpr int kDeflateWarp = round128(DeflateRing::SMEM + DeflateSmem::BYTES);
constexpr int kBatchWarp =
    round128(RleRing::SMEM + cmax(DeflateSmem::BYTES, cmax(kRleV1Scratch, kRleV2Scratch)));

struct Args {
  const uint8_t* comp;
  const uint64_t* comp_off;
  uint64_t n;
  uint8_t* out;
  const uint64_t* out_off;
  uint64_t* sizes;      // sizing kernels only
  int32_t* status;      // per chunk
  int format;           // plain kernels: the format of every chunk
  const uint8_t* formats;  // batch kernel: per-chunk format
  const uint32_t* order;   // batch kernel: claim order (may be null)
  uint32_t* counter;       // batch kernel: work counter (zeroed before launch)
};

// Plain kernels (one warp per chunk) and sizing kernels, per format family.
__global__ void rle_v1_kernel(Args a);
__global__ void rle_v1_sizes_kernel(Args a);
__global__ void rle_v2_kernel(Args a);
__global__ void rle_v2_sizes_kernel(Args a);
__global__ void inflate_kernel(Args a);
__global__ void inflate_sizes_kernel(Args a);

__global__ void batch_kernel(Args a);

// descending-size claim order for the batch kernel (counting sort by
// log2(compressed + uncompressed bytes)); hist/cursor are 64 words each
__global__ void order_hist_kernel(const uint64_t* comp_off, const uint64_t* out_off, uint64_t n,
                                  uint32_t* hist);
__global__ void order_scatter_kernel(const uint64_t* comp_off, const uint64_t* out_off,
                                     uint64_t n, const uint32_t* hist, uint32_t* cursor,
                                     uint32_t* order);

}  // namespace codag
