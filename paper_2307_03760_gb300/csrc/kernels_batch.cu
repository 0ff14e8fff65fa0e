// Persistent work-stealing kernel for mixed-format batches, the largest-first
// claim order it uses, and the status combination of multi-part chunks.
#include "batch.cuh"

namespace codag {

__global__ void order_hist_kernel(const uint8_t* formats, const uint64_t* comp_off,
                                  const uint64_t* out_off, uint64_t n, uint32_t* hist) {
  __shared__ uint32_t h[kBuckets];
  for (int i = threadIdx.x; i < kBuckets; i += blockDim.x) h[i] = 0;
  __syncthreads();
  for (uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n;
       c += (uint64_t)gridDim.x * blockDim.x)
    atomicAdd(&h[batch_bucket(formats, comp_off, out_off, c)], 1u);
  __syncthreads();
  for (int i = threadIdx.x; i < kBuckets; i += blockDim.x)
    if (h[i]) atomicAdd(&hist[i], h[i]);
}

__global__ void order_scatter_kernel(const uint8_t* formats, const uint64_t* comp_off,
                                     const uint64_t* out_off, uint64_t n, const uint32_t* hist,
                                     uint32_t* cursor, uint32_t* order) {
  __shared__ uint32_t start[kBuckets];
  if (threadIdx.x == 0) {
    uint32_t s = 0;
    for (int k = 0; k < kBuckets; k++) {
      start[k] = s;
      s += hist[k];
    }
  }
  __syncthreads();
  for (uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n;
       c += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t k = batch_bucket(formats, comp_off, out_off, c);
    order[start[k] + atomicAdd(&cursor[k], 1u)] = (uint32_t)c;
  }
}

__global__ void batch_finalize_kernel(const uint8_t* formats, const uint64_t* comp_off,
                                      const uint64_t* out_off, uint64_t n,
                                      const unsigned long long* keys, int32_t* status,
                                      uint32_t split_lg, uint32_t split_max) {
  for (uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n;
       c += (uint64_t)gridDim.x * blockDim.x)
    if (bucket_parts(batch_bucket(formats, comp_off, out_off, c), split_lg, split_max) > 1)
      status[c] = key_status(keys[c]);
}

CODAG_BATCH_SHAPE(1024, 4)

BatchShape batch_shape(int i) {
  switch (i) {
    case 0: return batch_shape_256x8();
    case 1: return batch_shape_512x8();
    case 2: return batch_shape_1024x4();
    case 3: return batch_shape_2048x4();
    default: return BatchShape{0, 0, nullptr, 0};
  }
}

// this unit's copy of the work-wait bound (codag_set_wait_limit_ns)
cudaError_t set_wait_limit_batch(uint64_t ns) { return set_wait_limit_here(ns); }

}  // namespace codag
