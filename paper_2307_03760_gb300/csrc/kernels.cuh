// Kernel entry points and their per-warp shared-memory layouts.
//
// Work mapping (CODAG Sec. II-B and IV-C): every chunk is independent; one
// warp decodes one chunk.  The plain kernels launch one warp per chunk and
// let the block scheduler hand out chunks; the batch kernel is persistent
// (one wave of CTAs) and its warps claim chunks with an atomic counter in
// descending-size order, so a mixed batch of uneven chunks keeps every SM busy
// and the largest chunks start first.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "byte_rle.cuh"
#include "inflate.cuh"
#include "rle_v1.cuh"
#include "rle_v2.cuh"

namespace codag {

constexpr int kWarpsPerBlock = 4;
constexpr int kThreads = 32 * kWarpsPerBlock;

using RleRing = InRing<1024, 4>;
using DeflateRing = InRing<256, 4>;
constexpr int kLitTB = 10, kDistTB = 8, kWin = 0;
using DeflateSmem = InflateSmem<kLitTB, kDistTB, kWin>;

__host__ __device__ constexpr int round128(int x) { return (x + 127) & ~127; }
constexpr int cmax(int a, int b) { return a > b ? a : b; }

constexpr int kRleV1Warp = round128(RleRing::SMEM + kRleV1Scratch);
constexpr int kRleV2Warp = round128(RleRing::SMEM + kRleV2Scratch);
constexpr int kDeflateWarp = round128(DeflateRing::SMEM + DeflateSmem::BYTES);
// per-warp shared memory of a one-warp-per-chunk kernel: input ring + scratch
// (Deflate tables for Deflate and ORC zlib streams; none for byte RLE)
__host__ __device__ constexpr int warp_chunk_smem(int family, int ring_smem) {
  return round128(ring_smem + (family == 4 ? 0 : DeflateSmem::BYTES));
}
// per-warp scratch of the RLE decoders besides their input
constexpr int kRleScratch = 512;
// plain RLE kernels: the smallest whole-chunk staging area per CTA (the
// launch widens it to the shared memory that occupancy leaves free)
constexpr int kRleStageBytes = 32768 + 256;
// segments of a staged RLE chunk: about kSegValues values each, at most kMaxSeg
constexpr int kMaxSeg = 64;
constexpr int kSegValues = 1024;
constexpr int kSegValuesV1 = 256;  // RLE v1: a cheap walk, so finer segments
constexpr int kSegBytesByteRle = 2048;  // byte / boolean RLE: decoded bytes per segment
// per-CTA extras: mbarrier, status key, published/claimed, split positions,
// counts and targets
constexpr int kRleCtaExtra = 24 + 3 * (kMaxSeg + 1) * 8;
// RLE v1 staged chunks add, after the extra region, a terminator bitmap of
// the stage and its rank directory (one word per 32 stage bytes plus 32 words
// of read slack each) and one word per warp for the rank totals.
__host__ __device__ constexpr int rle_v1_bitmap_words(int stage_bytes) { return stage_bytes / 32 + 32; }
__host__ __device__ constexpr int rle_v1_bitmap_bytes(int stage_bytes) { return (2 * rle_v1_bitmap_words(stage_bytes) + 32) * 4; }
constexpr int kRleMaxSmem = 16 * RleRing::SMEM + 16 * kRleScratch + kRleCtaExtra +
                            rle_v1_bitmap_bytes(16 * RleRing::SMEM);
// Deflate in the batch kernel may keep recent output in a shared window
// (kBatchWin bytes, 0 = none).  Measured on the 20,000-chunk mixed batch: an
// 8 or 16 KiB window halves throughput (fewer CTAs fit), so none is used.
constexpr int kBatchWin = 0;
using BatchDeflateSmem = InflateSmem<kLitTB, kDistTB, kBatchWin>;
// RLE decoders ask their input ring for spans of up to 1,608 bytes (an RLE v2
// run of 512 values of 25 bits, plus 8); every ring they read must cover that.
constexpr int kRleMinSpan = 1664;
static_assert(RleRing::MAX_SPAN >= kRleMinSpan, "RLE ring too shallow");
// Per-warp shared memory of the batch kernel with input ring Ring: the ring
// and the largest decoder scratch.
template <class Ring>
__host__ __device__ constexpr int batch_warp_bytes() {
  return round128(Ring::SMEM + cmax(BatchDeflateSmem::BYTES, cmax(kRleV1Scratch, kRleV2Scratch)));
}

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
  const uint32_t* order;   // batch kernel: chunks in claim order
  uint32_t* counter;       // batch kernel: kBatchCounterWords words, zeroed before launch
  unsigned long long* keys;  // batch kernel: combined status of multi-part chunks
  int stage_bytes;           // plain RLE kernels: shared staging area per CTA
  int deferred_only;         // one-warp Deflate kernel: decode only chunks whose status is kDeferred
  uint32_t split_lg;         // batch kernel: RLE split rule (bucket_parts)
  uint32_t split_max;
  // plain RLE v2 with a separate walk pass: kMaxSeg entries per chunk (see
  // rle_seg_count); entry 0 .x = 1 when the walk pass wrote the chunk's
  // segment starts, entries k = 1 .. nseg-1 = (stream position, value index)
  uint2* seg;
  int parts;  // warps per CTA of the decode pass the walk pass serves
};

// Batch scratch: [0] task counter, [1..128] bucket histogram, [129..256]
// bucket cursors.  Buckets order chunks largest first (2 * (63 - log2 of
// compressed + uncompressed bytes) + 1 for Deflate); an RLE chunk of 2^b
// bytes is split into min(2^(b - split_lg), split_max) parts when b >
// split_lg, else decoded whole (the default rule: split_lg 16, split_max 16).
constexpr int kBuckets = 128;
constexpr int kBatchCounterWords = 1 + 2 * kBuckets;

__host__ __device__ __forceinline__ bool is_rle_format(int f) {
  return f == FMT_RLE_V1_I64 || f == FMT_RLE_V1_U64 || f == FMT_RLE_V2_I64 || f == FMT_RLE_V2_U64;
}

__device__ __forceinline__ uint32_t batch_bucket(const uint8_t* formats, const uint64_t* comp_off,
                                                 const uint64_t* out_off, uint64_t c) {
  const uint64_t b = (comp_off[c + 1] - comp_off[c]) + (out_off[c + 1] - out_off[c]);
  const uint32_t lg = 63u - (uint32_t)__clzll((long long)(b | 1));
  return 2u * (63u - lg) + (is_rle_format(formats[c]) ? 0u : 1u);
}

constexpr uint32_t kSplitLgDefault = 16, kSplitMaxDefault = 16, kSplitMaxLimit = 32;

__host__ __device__ __forceinline__ uint32_t bucket_parts(uint32_t bucket, uint32_t split_lg,
                                                          uint32_t split_max) {
  if (bucket & 1u) return 1u;
  const uint32_t lg = 63u - (bucket >> 1);
  if (lg <= split_lg) return 1u;
  const uint32_t d = lg - split_lg;
  const uint32_t p = d >= 6 ? 64u : (1u << d);
  return p < split_max ? p : split_max;
}

// Plain kernels.  RLE: one CTA per chunk, blockDim.x / 32 warps decoding its
// parts, dynamic shared memory = warps * per-warp size + 16.  Deflate: one
// warp per chunk, kWarpsPerBlock warps per CTA.  *_sizes_* decode without
// storing and write each chunk's decoded size (RLE: one warp per CTA).
__global__ void orc_zlib_kernel(Args a);
__global__ void orc_zlib_sizes_kernel(Args a);
__global__ void byte_rle_kernel(Args a);
__global__ void byte_rle_cta_kernel(Args a);
__global__ void byte_rle_reg_kernel(Args a);
__global__ void inflate_reg_kernel(Args a);
__global__ void byte_rle_sizes_kernel(Args a);
__global__ void rle_v1_kernel(Args a);
__global__ void rle_v1_sizes_kernel(Args a);
__global__ void rle_v2_kernel(Args a);
__global__ void rle_v2_sizes_kernel(Args a);
// Walk pass of the plain RLE v2 call: one warp per chunk (kWarpsPerBlock per
// CTA) walks the run headers of every chunk that the decode pass stages
// whole and writes its segment starts to a.seg.
__global__ void rle_v2_walk_kernel(Args a);
__global__ void inflate_kernel(Args a);
__global__ void inflate_sizes_kernel(Args a);

// Two-pass raw Deflate (inflate_lanes.cuh): Huffman decoding with one lane
// per chunk (persistent CTAs of kHufWarps warps, chunks claimed through
// h.counter), then the LZ77 copies with one warp per chunk.  The sizes
// kernel runs the first pass alone, without output or commands.
struct HufArgs;
__global__ void inflate_huffman_kernel(Args a, HufArgs h);
__global__ void inflate_huffman_sizes_kernel(Args a, HufArgs h);
__global__ void inflate_lz77_kernel(Args a, HufArgs h);

// Persistent batch kernel (batch.cuh): warps claim (chunk, part) tasks in
// bucket order, each warp reading its input through a shared-memory ring of
// SLOT x SLOTS bytes.  It is compiled for kBatchShapes ring shapes and one is
// chosen at launch (codag_set_batch_staging).
struct BatchShape {
  int slot;        // bytes per ring slot
  int slots;       // slots per ring
  const void* fn;  // the kernel instance
  int smem;        // its dynamic shared memory per CTA
};
constexpr int kBatchShapes = 4;
constexpr int kBatchShapeDefault = 2;  // 1024 x 4
BatchShape batch_shape(int i);  // i in [0, kBatchShapes): 256x8, 512x8, 1024x4, 2048x4
BatchShape batch_shape_256x8();
BatchShape batch_shape_512x8();
BatchShape batch_shape_1024x4();
BatchShape batch_shape_2048x4();

// claim order for the batch kernel (counting sort by bucket)
__global__ void order_hist_kernel(const uint8_t* formats, const uint64_t* comp_off,
                                  const uint64_t* out_off, uint64_t n, uint32_t* hist);
__global__ void order_scatter_kernel(const uint8_t* formats, const uint64_t* comp_off,
                                     const uint64_t* out_off, uint64_t n, const uint32_t* hist,
                                     uint32_t* cursor, uint32_t* order);
// status of multi-part chunks from their combined keys
__global__ void batch_finalize_kernel(const uint8_t* formats, const uint64_t* comp_off,
                                      const uint64_t* out_off, uint64_t n,
                                      const unsigned long long* keys, int32_t* status,
                                      uint32_t split_lg, uint32_t split_max);

// Host: set the work-wait bound (codag_set_wait_limit_ns) in each unit that
// has bounded device waits.
cudaError_t set_wait_limit_rle(uint64_t ns);
cudaError_t set_wait_limit_inflate(uint64_t ns);
cudaError_t set_wait_limit_batch(uint64_t ns);
cudaError_t set_wait_limit_batch_small(uint64_t ns);
cudaError_t set_wait_limit_batch_large(uint64_t ns);

// Dynamic shared memory of the batch kernel with input ring Ring: per-warp
// regions + bucket tables.
template <class Ring>
__host__ __device__ constexpr int batch_smem() {
  return kWarpsPerBlock * batch_warp_bytes<Ring>() + 2 * (kBuckets + 1) * 4;
}

}  // namespace codag
