// Persistent work-stealing kernel for mixed-format batches, the largest-first
// claim order it uses, and the status combination of multi-part chunks.
#include "chunk.cuh"

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
                                      const unsigned long long* keys, int32_t* status) {
  for (uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n;
       c += (uint64_t)gridDim.x * blockDim.x)
    if (bucket_parts(batch_bucket(formats, comp_off, out_off, c)) > 1) status[c] = key_status(keys[c]);
}

__global__ void __launch_bounds__(kThreads) batch_kernel(Args a) {
  extern __shared__ __align__(128) uint8_t smem[];
  uint32_t* tstart = reinterpret_cast<uint32_t*>(smem + kWarpsPerBlock * kBatchWarp);
  uint32_t* cstart = tstart + kBuckets + 1;
  if (threadIdx.x == 0) {
    const uint32_t* hist = a.counter + 1;
    uint32_t t = 0, cc = 0;
    for (int b = 0; b < kBuckets; b++) {
      tstart[b] = t;
      cstart[b] = cc;
      t += hist[b] * bucket_parts((uint32_t)b);
      cc += hist[b];
    }
    tstart[kBuckets] = t;
    cstart[kBuckets] = cc;
  }
  __syncthreads();
  const uint32_t total = tstart[kBuckets];
  const uint32_t warp = threadIdx.x >> 5;
  uint8_t* region = smem + warp * kBatchWarp;
  uint8_t* scratch = region + RleRing::SMEM;
  RleRing ring;
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
    const uint32_t parts = bucket_parts((uint32_t)lo);
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
      r = decode_part<3, true, RleRing, kBatchWin>(ring, scratch, a, c, f, 0, 1);
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

// this unit's copy of the work-wait bound (codag_set_wait_limit_ns)
cudaError_t set_wait_limit_batch(uint64_t ns) { return set_wait_limit_here(ns); }

}  // namespace codag
