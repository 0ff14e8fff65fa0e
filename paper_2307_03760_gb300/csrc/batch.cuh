// The persistent batch kernel, a template over its per-warp input ring.
// Each translation unit that instantiates a ring shape defines that shape's
// launch record with CODAG_BATCH_SHAPE (kernels_batch*.cu).
#pragma once

#include "chunk.cuh"

namespace codag {

// Warps claim (chunk, part) tasks from one counter in bucket order (largest
// first); an RLE chunk of bucket b is cut into bucket_parts(b) parts, each
// decoded by the warp that claims it after walking to the part's start.
template <class Ring>
__global__ void __launch_bounds__(kThreads, 1) batch_kernel(Args a) {
  static_assert(Ring::MAX_SPAN >= kRleMinSpan, "batch ring too shallow for the RLE decoders");
  constexpr int kWarpBytes = batch_warp_bytes<Ring>();
  extern __shared__ __align__(128) uint8_t smem[];
  uint32_t* tstart = reinterpret_cast<uint32_t*>(smem + kWarpsPerBlock * kWarpBytes);
  uint32_t* cstart = tstart + kBuckets + 1;
  if (threadIdx.x == 0) {
    const uint32_t* hist = a.counter + 1;
    uint32_t t = 0, cc = 0;
    for (int b = 0; b < kBuckets; b++) {
      tstart[b] = t;
      cstart[b] = cc;
      t += hist[b] * bucket_parts((uint32_t)b, a.split_lg, a.split_max);
      cc += hist[b];
    }
    tstart[kBuckets] = t;
    cstart[kBuckets] = cc;
  }
  __syncthreads();
  const uint32_t total = tstart[kBuckets];
  const uint32_t warp = threadIdx.x >> 5;
  uint8_t* region = smem + warp * kWarpBytes;
  uint8_t* scratch = region + Ring::SMEM;
  Ring ring;
  ring.init(region);
  for (;;) {
    uint32_t t = 0;
    if (lane_id() == 0) t = atomicAdd(a.counter, 1u);
    t = __shfl_sync(FULL, t, 0);
    if (t >= total) break;
    int lo = 0, hi = kBuckets;  // largest b with tstart[b] <= t
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (tstart[mid] <= t) lo = mid;
      else hi = mid;
    }
    const uint32_t parts = bucket_parts((uint32_t)lo, a.split_lg, a.split_max);
    const uint32_t rel = t - tstart[lo];
    const uint64_t c = a.order[cstart[lo] + rel / parts];
    const uint32_t part = rel % parts;
    const int f = a.formats[c];
    PartResult r;
    if (f == FMT_RLE_V1_I64 || f == FMT_RLE_V1_U64)
      r = decode_part<1, true>(ring, scratch, a, c, f, part, parts);
    else if (f == FMT_RLE_V2_I64 || f == FMT_RLE_V2_U64)
      r = decode_part<2, true>(ring, scratch, a, c, f, part, parts);
    else if (f == FMT_DEFLATE)
      r = decode_part<3, true, Ring, kBatchWin>(ring, scratch, a, c, f, 0, 1);
    else if (f == FMT_BYTE_RLE || f == FMT_BOOL_RLE)
      r = decode_part<4, true>(ring, scratch, a, c, f, 0, 1);
    else if (f == FMT_ORC_ZLIB)
      r = decode_part<5, true>(ring, scratch, a, c, f, 0, 1);
    else
      r = PartResult{ST_BAD_HEADER, 0, 0};
    if (lane_id() == 0) {
      if (parts == 1) a.status[c] = r.status;
      else if (r.status != ST_OK) atomicMin(&a.keys[c], status_key(r));
    }
    if (r.status == ST_TIMEOUT) break;  // this warp's ring state is no longer trusted
  }
}


#define CODAG_BATCH_SHAPE(SLOT, SLOTS)                                                  \
  BatchShape batch_shape_##SLOT##x##SLOTS() {                                           \
    using R = InRing<SLOT, SLOTS>;                                                      \
    return BatchShape{SLOT, SLOTS, (const void*)batch_kernel<R>, batch_smem<R>()};      \
  }

}  // namespace codag
