// One chunk, end to end, for any format: bounds checks on the offsets
// metadata (CODAG Sec. II-B: each chunk is located by its compressed and
// uncompressed offsets), staging-ring start, the format decoder, and the
// drain of in-flight staging copies.
#pragma once

#include "kernels.cuh"

namespace codag {

// Decode (STORE) or size (!STORE) chunk c with the decoder of `family`.
// Returns the chunk status; *produced = output bytes.
template <int FAMILY, bool STORE, class Ring>
__device__ __forceinline__ int32_t decode_chunk(Ring& ring, uint8_t* scratch, const Args& a,
                                                uint64_t c, int format, uint64_t* produced) {
  *produced = 0;
  const uint64_t total = a.comp_off[a.n];
  const uint64_t cs = a.comp_off[c], ce = a.comp_off[c + 1];
  if (ce < cs || ce > total) return ST_BAD_SPAN;
  uint64_t os = 0, cap = ~0ull;
  if (STORE) {
    os = a.out_off[c];
    const uint64_t oe = a.out_off[c + 1];
    if (oe < os) return ST_BAD_SPAN;
    cap = oe - os;
    if (FAMILY != 3 && ((cap & 7) || (os & 7))) return ST_BAD_SPAN;
  }
  const int64_t n_in = (int64_t)(ce - cs);
  ring.start(a.comp + cs, n_in, a.comp + total);
  int32_t st;
  uint64_t prod = 0;
  if (FAMILY == 1) {
    const bool sgn = format == FMT_RLE_V1_I64;
    st = rle_v1_decode<STORE>(ring, reinterpret_cast<uint16_t*>(scratch), n_in, sgn,
                              reinterpret_cast<uint64_t*>(a.out + os), cap / 8, &prod);
    prod *= 8;
  } else if (FAMILY == 2) {
    const bool sgn = format == FMT_RLE_V2_I64;
    st = rle_v2_decode<STORE>(ring, scratch, n_in, sgn, reinterpret_cast<uint64_t*>(a.out + os),
                              cap / 8, &prod);
    prod *= 8;
  } else {
    st = inflate_decode<STORE, kLitTB, kDistTB, kWin>(ring, scratch, n_in, a.out + os, cap, &prod);
  }
  // bounded wait for this warp's own copies still in flight, also after a timeout
  if (!ring.drain()) st = ST_TIMEOUT;
  *produced = prod;
  return st;
}

// Body of the plain kernels: one warp per chunk, one chunk per warp.
template <int FAMILY, bool STORE, int PER_WARP, class Ring>
__device__ __forceinline__ void chunk_body(const Args& a) {
  extern __shared__ __align__(128) uint8_t smem[];
  const uint32_t warp = threadIdx.x >> 5;
  const uint64_t c = (uint64_t)blockIdx.x * kWarpsPerBlock + warp;
  if (c >= a.n) return;
  uint8_t* region = smem + warp * PER_WARP;
  Ring ring;
  ring.init(region);
  uint64_t produced;
  const int32_t st = decode_chunk<FAMILY, STORE>(ring, region + Ring::SMEM, a, c, a.format, &produced);
  if (lane_id() == 0) {
    a.status[c] = st;
    if (!STORE) a.sizes[c] = produced;
  }
}

}  // namespace codag
