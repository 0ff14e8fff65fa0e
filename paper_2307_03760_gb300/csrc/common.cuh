// Shared device primitives for the chunk decoders (sm_103a).
//
// A "decoder" is one warp that owns one compressed chunk at a time (CODAG
// Sec. IV-C: the decompression unit is a warp, every lane follows the same
// control flow and holds the same decoding state, Sec. IV-D).  This file holds
// what all formats share: per-chunk status codes, PTX wrappers for the 1-D
// TMA bulk copy and mbarriers used by the input staging ring, and small
// bit/byte helpers.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace codag {

// Per-chunk status codes (the values are part of the C ABI, include/codag.h).
enum ChunkStatus : int32_t {
  ST_OK = 0,
  ST_TRUNCATED = 1,
  ST_OVERFLOW = 2,
  ST_UNDERFLOW = 3,
  ST_BAD_HEADER = 4,
  ST_BAD_HUFFMAN = 5,
  ST_BAD_DISTANCE = 6,
  ST_BAD_STORED_LEN = 7,
  ST_BAD_SPAN = 8,
  ST_TIMEOUT = 9,
};
// Internal status (never returned): a Deflate chunk the two-pass decoder
// left to the one-warp decoder, which then writes its final status.
constexpr int32_t kDeferred = 0x40;

// Format identifiers (C ABI values).
enum Format : int {
  FMT_RLE_V1_I64 = 1,
  FMT_RLE_V2_I64 = 2,
  FMT_DEFLATE = 3,
  FMT_RLE_V1_U64 = 4,
  FMT_RLE_V2_U64 = 5,
  FMT_BYTE_RLE = 6,
  FMT_BOOL_RLE = 7,
  FMT_ORC_ZLIB = 8,
};

constexpr unsigned FULL = 0xffffffffu;

// Result of decoding one part of a chunk: status, the stream position of the
// run or group where it was found (errors of several parts are combined by
// taking the earliest position, which is the first error in stream order),
// and the values walked.
struct PartResult {
  int32_t status;
  int64_t err_pos;
  uint64_t count;
};

__device__ __forceinline__ PartResult part_error(int32_t st, int64_t pos, uint64_t count) {
  return PartResult{st, pos, count};
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ uint64_t unzigzag(uint64_t u) { return (u >> 1) ^ (0ull - (u & 1)); }

__device__ __forceinline__ uint64_t bswap64(uint64_t x) {
  uint32_t lo = (uint32_t)x, hi = (uint32_t)(x >> 32);
  return ((uint64_t)__byte_perm(lo, 0, 0x0123) << 32) | __byte_perm(hi, 0, 0x0123);
}

__device__ __forceinline__ uint32_t bswap32(uint32_t x) { return __byte_perm(x, 0, 0x0123); }

// low `n` bits set, 0 <= n <= 64
__device__ __forceinline__ uint64_t lowmask64(uint32_t n) {
  return n >= 64 ? ~0ull : ((1ull << n) - 1);
}

__device__ __forceinline__ uint64_t shfl64(uint64_t v, int src) {
  uint32_t lo = __shfl_sync(FULL, (uint32_t)v, src);
  uint32_t hi = __shfl_sync(FULL, (uint32_t)(v >> 32), src);
  return ((uint64_t)hi << 32) | lo;
}

__device__ __forceinline__ uint64_t shfl_up64(uint64_t v, int d) {
  uint32_t lo = __shfl_up_sync(FULL, (uint32_t)v, d);
  uint32_t hi = __shfl_up_sync(FULL, (uint32_t)(v >> 32), d);
  return ((uint64_t)hi << 32) | lo;
}

// inclusive prefix sum (mod 2^32) across the warp
__device__ __forceinline__ uint32_t warp_incl_scan32(uint32_t v) {
  const uint32_t lane = lane_id();
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t t = __shfl_up_sync(FULL, v, d);
    if (lane >= (uint32_t)d) v += t;
  }
  return v;
}

// inclusive prefix sum (mod 2^64) across the warp
__device__ __forceinline__ uint64_t warp_incl_scan64(uint64_t v) {
  const uint32_t lane = lane_id();
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    uint64_t t = shfl_up64(v, d);
    if (lane >= (uint32_t)d) v += t;
  }
  return v;
}

// ------------------------------------------------------------------ PTX ---
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (TMA) accesses.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

// 1-D bulk copy global -> shared (TMA); completion is signalled on `bar` as
// transaction bytes.  dst and src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Test a phase; the thread may be suspended (up to about 0.1 ms, the time
// hint) until the phase completes, so waiting costs few instructions.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity), "r"(100000u)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Test a phase without waiting.
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounds on one mbarrier phase wait before the decoder gives up on the chunk
// (ST_TIMEOUT): wall time, and a poll count in case the timer stalls.  A TMA
// copy of at most a few KiB completes in microseconds.
constexpr uint64_t kMaxWaitNs = 100ull * 1000 * 1000;  // 100 ms
constexpr uint32_t kMaxWaitPolls = 1u << 20;

// Bound of a wait on work in progress (a copy the decoder needs next, a
// segment start another warp publishes): kMaxWaitNs unless
// codag_set_wait_limit_ns shortens it (0: give up unless already complete),
// so that tests can make such waits run out.  A decoder's wait for its own
// copies in flight before it stops always uses kMaxWaitNs.  One copy per
// translation unit, set through set_wait_limit_here().
static __device__ uint64_t g_wait_limit_ns = kMaxWaitNs;

__device__ __forceinline__ uint64_t work_wait_ns() {
  return *reinterpret_cast<volatile uint64_t*>(&g_wait_limit_ns);
}

// Wait for `parity` of `bar` for at most limit_ns; false if the wait ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  uint64_t limit_ns = kMaxWaitNs) {
  if (limit_ns == 0) return mbar_test(bar, parity);
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  for (uint32_t polls = 0; polls < kMaxWaitPolls; polls++) {
    if (mbar_try_wait(bar, parity)) return true;
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
  return false;
}

// Host: this translation unit's copy of the work-wait bound.
static inline cudaError_t set_wait_limit_here(uint64_t ns) {
  return cudaMemcpyToSymbol(g_wait_limit_ns, &ns, sizeof(ns));
}

}  // namespace codag
