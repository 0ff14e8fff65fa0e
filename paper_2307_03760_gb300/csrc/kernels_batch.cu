// Persistent work-stealing kernel for mixed-format batches, and the
// descending-size claim order it uses.
#include "chunk.cuh"

namespace codag {

__device__ __forceinline__ uint32_t size_class(const uint64_t* comp_off, const uint64_t* out_off,
                                               uint64_t c) {
  const uint64_t b = (comp_off[c + 1] - comp_off[c]) + (out_off[c + 1] - out_off[c]);
  return 63u - (uint32_t)(63 - __clzll((long long)(b | 1)));  // larger chunks -> smaller key
}

__global__ void order_hist_kernel(const uint64_t* comp_off, const uint64_t* out_off, uint64_t n,
                                  uint32_t* hist) {
  __shared__ uint32_t h[64];
  if (threadIdx.x < 64) h[threadIdx.x] = 0;
  __syncthreads();
  for (uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n;
       c += (uint64_t)gridDim.x * blockDim.x)
    atomicAdd(&h[size_class(comp_off, out_off, c)], 1u);
  __syncthreads();
  if (threadIdx.x < 64 && h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], h[threadIdx.x]);
}

__global__ void order_scatter_kernel(const uint64_t* comp_off, const uint64_t* out_off,
                                     uint64_t n, const uint32_t* hist, uint32_t* cursor,
                                     uint32_t* order) {
  __shared__ uint32_t start[64];
  if (threadIdx.x == 0) {
    uint32_t s = 0;
    for (int k = 0; k < 64; k++) {
      start[k] = s;
      s += hist[k];
    }
  }
  __syncthreads();
  for (uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n;
       c += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t k = size_class(comp_off, out_off, c);
    order[start[k] + atomicAdd(&cursor[k], 1u)] = (uint32_t)c;
  }
}

__global__ void __launch_bounds__(kThreads) batch_kernel(Args a) {
  extern __shared__ __align__(128) uint8_t smem[];
  const uint32_t warp = threadIdx.x >> 5;
  uint8_t* region = smem + warp * kBatchWarp;
  uint8_t* scratch = region + RleRing::SMEM;
  RleRing ring;
  ring.init(region);
  for (;;) {
    uint32_t idx = 0;
    if (lane_id() == 0) idx = atomicAdd(a.counter, 1u);
    idx = __shfl_sync(FULL, idx, 0);
    if ((uint64_t)idx >= a.n) break;
    const uint64_t c = a.order ? a.order[idx] : idx;
    const int f = a.formats[c];
    uint64_t produced;
    int32_t st;
    if (f == FMT_RLE_V1_I64 || f == FMT_RLE_V1_U64)
      st = decode_chunk<1, true>(ring, scratch, a, c, f, &produced);
    else if (f == FMT_RLE_V2_I64 || f == FMT_RLE_V2_U64)
      st = decode_chunk<2, true>(ring, scratch, a, c, f, &produced);
    else if (f == FMT_DEFLATE)
      st = decode_chunk<3, true>(ring, scratch, a, c, f, &produced);
    else
      st = ST_BAD_HEADER;
    if (lane_id() == 0) a.status[c] = st;
    if (st == ST_TIMEOUT) break;  // this warp's ring state is no longer trusted
  }
}

}  // namespace codag
